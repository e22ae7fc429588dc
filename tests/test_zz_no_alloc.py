"""The allocation-free block dot product (sg_block_dot_noalloc): for callers
that cannot call cudaMalloc (pool-allocator frameworks, fixed memory
budgets, code that must avoid cudaFree's device-wide synchronisation).

Its GPU test calls it through the C ABI on two calls in a row and checks the
result against sg_block_dot and against the FP64 definition W = Q^T X
formed on the host, within the block-dot tolerance of the parity tests.  One
shape needs more split partial sums than the fixed scratch holds, so the
call takes its reduced-split path.  This file is collected last so a
stop-at-first-failure run has already run the rest.
"""
import ctypes as C

import numpy as np
import pytest

import paper_2303_08953_gb300 as sg

SCRATCH_DOUBLES = 1 << 19   # SG_NOALLOC_SCRATCH_DOUBLES in include/sgmres.h


def test_noalloc_rejects_shapes_beyond_its_scratch():
    err = C.create_string_buffer(256)
    i, s = 1024, 1024  # i*s > SG_NOALLOC_SCRATCH_DOUBLES (2^19)
    rc = sg.lib.sg_block_dot_noalloc(10, None, 10, i, None, 10, s, None, i,
                                     None, err, 256)
    assert rc == sg.SG_EINVAL
    assert b"exceeds the scratch" in err.value


def _uncapped_splits(n, i, s, sms):
    """Split count the FP64 block dot picks when scratch is unlimited: one
    wave of 8 CTAs per SM over the output tiles (64 x 8 tiles for s <= 8),
    at most one split per 128 rows."""
    assert i > 8 and s <= 8
    tiles = -(-i // 64) * -(-s // 8)
    S = min((sms * 8) // tiles, -(-n // 128))
    rows = -(-(-(-n // S)) // 32) * 32     # rows per split, whole 32-row stages
    return -(-n // rows)


@pytest.mark.gpu
def test_noalloc_block_dot_matches_block_dot_and_definition_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    capped = (1 << 20, 64, 8)
    assert _uncapped_splits(*capped, sms) * 64 * 8 > SCRATCH_DOUBLES
    solver = sg.Solver(0)
    try:
        dev = torch.device("cuda:0")
        err = C.create_string_buffer(256)
        for call, (n, i, s) in enumerate([(70001, 121, 40), (70001, 121, 40),
                                          (4133, 3, 7), capped, capped]):
            rng = np.random.default_rng(700 + call)
            ld = n + 5
            Qh = rng.standard_normal((i, ld))
            Xh = rng.standard_normal((s, ld))
            Q = torch.as_tensor(Qh, device=dev)
            X = torch.as_tensor(Xh, device=dev)
            W_ref = torch.empty((s, i), dtype=torch.float64, device=dev)
            W_na = torch.full((s, i), float("nan"), dtype=torch.float64, device=dev)
            st = sg._stream_ptr()
            rc = sg.lib.sg_block_dot(solver._h, n, C.c_void_p(Q.data_ptr()), ld, i,
                                     C.c_void_p(X.data_ptr()), ld, s,
                                     C.c_void_p(W_ref.data_ptr()), i, 0, st)
            assert rc == 0
            rc = sg.lib.sg_block_dot_noalloc(n, C.c_void_p(Q.data_ptr()), ld, i,
                                             C.c_void_p(X.data_ptr()), ld, s,
                                             C.c_void_p(W_na.data_ptr()), i, st,
                                             err, 256)
            assert rc == 0, err.value
            torch.cuda.synchronize()
            a = W_na.cpu().numpy()
            b = W_ref.cpu().numpy()
            # W[c, r] = sum_k Q[r, k] X[c, k] over the n rows (the definition)
            d = Xh[:, :n] @ Qh[:, :n].T
            scale = np.abs(Xh[:, :n]) @ np.abs(Qh[:, :n]).T
            assert np.all(np.abs(a - b) <= 2e-14 * scale + 1e-300)
            assert np.all(np.abs(a - d) <= 2e-14 * scale + 1e-300)
            del Q, X
    finally:
        solver.close()
