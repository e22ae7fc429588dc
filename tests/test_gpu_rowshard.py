"""The row-partitioned solve (Alg. 4 over row blocks, Sec. 5) with the CUDA
kernels: two ranks, each a process driving the library on cuda:0, with
gloo collectives staged through host memory.  The ranks' kernels never
wait on one another (every exchange and reduction is a host collective
between kernel launches), so two processes can share the one GPU.  Same
bar as the CPU form: the oracle's decisions on every rank and x within
1e-9 of the oracle's."""
import numpy as np
import pytest

from test_rowshard import SYSTEMS, check_against_oracle, run_ranks

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)


@pytest.mark.parametrize("name", list(SYSTEMS))
def test_two_gpu_ranks_match_the_single_rank_oracle(name):
    res = run_ranks(name, 2, device_ops=True)
    check_against_oracle(name, res)
    assert np.array_equal(res[0]["x"], res[1]["x"])
