"""The allocation-free Davidson projection against the allocating one.

fnocc_multi_dot_noalloc serves callers that cannot allocate device memory
themselves (their device memory belongs to another allocator, or they must
avoid the device-wide synchronisation of cudaFree): it keeps its partial sums
in a fixed array of the library instead of context memory. Through the C ABI
it must give what fnocc_multi_dot gives, call after call, and refuse requests
beyond its fixed scratch (more than 64 vectors).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-10  # the max-abs tolerance of the FP64 parity tests


def test_noalloc_multi_dot_matches_allocating_entry():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2509_14157_gb300 as pkg
    lib = pkg.load_library()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(0)
    ctx = pkg.Context(0)
    for n, nvec, seed in [(100003, 17, 1), (5000, 64, 2)]:  # two calls in a row, different data
        ld = n + 5
        gen = torch.Generator().manual_seed(seed)
        x = torch.randn(n, dtype=torch.float64, generator=gen).to(dev)
        y = torch.randn(nvec * ld, dtype=torch.float64, generator=gen).to(dev)
        ref = torch.zeros(nvec, dtype=torch.float64, device=dev)
        got = torch.full((nvec,), float("nan"), dtype=torch.float64, device=dev)
        torch.cuda.synchronize()
        ctx.multi_dot_dev(x.data_ptr(), y.data_ptr(), n, ld, nvec, ref.data_ptr())
        st = lib.fnocc_multi_dot_noalloc(x.data_ptr(), y.data_ptr(), n, ld, nvec, got.data_ptr(), None)
        assert st == 0
        torch.cuda.synchronize()
        r, g = ref.cpu().numpy(), got.cpu().numpy()
        assert np.all(np.isfinite(g))
        assert np.max(np.abs(g - r)) < TOL
        exact = (y.view(nvec, ld)[:, :n].cpu().numpy() @ x.cpu().numpy())
        assert np.max(np.abs(g - exact)) < 1e-9 * max(1.0, np.max(np.abs(exact)))
    # beyond the fixed scratch: rejected, output untouched
    out = torch.zeros(65, dtype=torch.float64, device=dev)
    big = torch.zeros(65 * 16, dtype=torch.float64, device=dev)
    torch.cuda.synchronize()
    st = lib.fnocc_multi_dot_noalloc(big.data_ptr(), big.data_ptr(), 16, 16, 65, out.data_ptr(), None)
    assert st == -1
    ctx.close()
