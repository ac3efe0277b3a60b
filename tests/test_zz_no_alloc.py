"""ffb_polar_noalloc: the polar transform without device allocation.

Some callers cannot call cudaMalloc where they run this step: code executed
while a stream is captured into a CUDA graph (allocation is illegal there),
serving loops with a fixed latency budget, and frameworks that hand out all
device memory from their own pool.  For them the library keeps a static
16 MiB scratch array per device instead of the plan's allocated scratch.

The test calls the entry point through the C ABI twice in a row on fresh
inputs and compares each result with ffb_polar (the allocating entry point)
at the tolerance of the other parity tests; it also checks that the second
call leaves PyTorch's allocator untouched and takes no device memory (free
memory does not drop by a 2 MiB allocation granule; other work on the device
could move it by less).  It sorts last in collection
so that a failure here cannot stop the rest of a -x run, and it builds the
library itself so that it also passes when run alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1412_0781_gb300 import ffb
    return ffb.load()


@pytest.mark.parametrize("L,n", [(64, 301), (128, 90)])
def test_polar_noalloc_matches_polar_on_two_calls(lib, L, n):
    from paper_1412_0781_gb300 import Plan, data
    dev = torch.device("cuda:0")
    plan = Plan(L, 0.5, L / 2, eps=1e-6)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    shape = (n, plan.n_xi, plan.n_theta // 2, 2)
    out = torch.empty(shape, device=dev, dtype=torch.float32)
    for call in range(2):
        x = data.white_noise(n, L, seed=4242 + 17 * call + L, device=dev)
        ref = plan.polar(x)
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        torch_before = (torch.cuda.memory_allocated(dev), torch.cuda.memory_reserved(dev))
        rc = lib.ffb_polar_noalloc(plan.handle, ctypes.c_void_p(x.data_ptr()), n,
                                   ctypes.c_void_p(out.data_ptr()), stream)
        assert rc == 0, rc
        torch.cuda.synchronize()
        plan.sync()
        if call == 1:
            assert (torch.cuda.memory_allocated(dev), torch.cuda.memory_reserved(dev)) == torch_before
            assert torch.cuda.mem_get_info()[0] > free_before - (2 << 20)
        a = out.double().cpu().numpy()
        b = ref.double().cpu().numpy()
        assert np.linalg.norm(a - b) / np.linalg.norm(b) <= TOL
    plan.close()
