"""sbd_fft2_noalloc: the allocation-free 2-D FFT agrees with sbd_fft2.

For callers that cannot allocate device memory while running (their memory is all
held by their own pool, or their policy forbids cudaMalloc after start-up), the
library offers one entry point whose scratch lives in a fixed device array.  This
file is collected last so that, if it fails, a run stopping at the first failure
has already run every other test; it passes alone and after the other tests.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1711_07877_gb300 import build
    build.build_library()
    import paper_1711_07877_gb300 as pkg
    return pkg


def _dev(x, dtype):
    return torch.from_numpy(x).to(dtype).cuda()


@pytest.mark.parametrize("form,shape", [(0, (64, 80)), (0, (512, 512)), (1, (500, 1024)), (1, (30, 4000))])
def test_noalloc_matches_allocating_fft2_twice(S, form, shape):
    dtype = torch.complex64 if form == 1 else torch.complex128
    tol = 2e-6 if form == 1 else 1e-12            # the FFT parity tolerances of test_gpu_parity.py
    rng = np.random.default_rng(sum(shape) + 7 * form)
    for call in range(2):                          # two calls in a row share the scratch array
        sign = -1 if call == 0 else 1
        x = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
        xt = _dev(x, dtype)
        ref = torch.empty_like(xt)
        S.sbd_fft2(xt, ref, shape[0], shape[1], sign, form)
        got = torch.empty_like(xt)
        S.sbd_fft2_noalloc(xt, got, shape[0], shape[1], sign, form)
        torch.cuda.synchronize()
        rel = (torch.linalg.norm(got - ref) / torch.linalg.norm(ref)).item()
        assert rel <= tol, (call, rel)


def test_noalloc_in_place_and_at_its_limits(S):
    """in and out may alias; 64 x 4096 FP64 fills the array exactly (4 MiB) at the largest
    side, where the row kernel holds a 64 KB FP64 row."""
    for form, shape in [(0, (64, 4096)), (1, (4096, 128)), (0, (48, 50))]:
        dtype = torch.complex64 if form == 1 else torch.complex128
        tol = 2e-6 if form == 1 else 1e-12
        rng = np.random.default_rng(shape[0] + shape[1])
        x = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
        xt = _dev(x, dtype)
        ref = torch.empty_like(xt)
        S.sbd_fft2(xt, ref, shape[0], shape[1], -1, form)
        S.sbd_fft2_noalloc(xt, xt, shape[0], shape[1], -1, form)     # in place
        torch.cuda.synchronize()
        rel = (torch.linalg.norm(xt - ref) / torch.linalg.norm(ref)).item()
        assert rel <= tol, (shape, rel)


def test_noalloc_rejects_sizes_beyond_its_array(S):
    big = torch.zeros(1024, 1024, dtype=torch.complex128, device="cuda")   # 16 MiB > 4 MiB
    with pytest.raises(S.SbdError) as e:
        S.sbd_fft2_noalloc(big, big, 1024, 1024, -1, 0)
    assert e.value.code == S.SBD_EINVAL
    over = torch.zeros(80, 4096, dtype=torch.complex128, device="cuda")   # valid sides, 5 MiB
    with pytest.raises(S.SbdError) as e:
        S.sbd_fft2_noalloc(over, over, 80, 4096, -1, 0)
    assert e.value.code == S.SBD_EINVAL
    side = torch.zeros(2, 5000, dtype=torch.complex64, device="cuda")
    with pytest.raises(S.SbdError) as e:
        S.sbd_fft2_noalloc(side, side, 2, 5000, -1, 1)
    assert e.value.code == S.SBD_EINVAL
