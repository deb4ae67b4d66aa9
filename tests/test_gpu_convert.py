"""The library's binary64 <-> binary32 conversions (integer operations on the
bit patterns, used on the FP64 residual and the FP64 correction of the
mixed-precision V-cycle) against the hardware conversion: bit-identical on
random values over the whole exponent range, exact ties (round half to even),
values that round up into the next binade, overflow, float subnormals, zeros,
infinities and NaN."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_1512_02390_gb300")


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P.load_library()


def _doubles():
    rng = np.random.default_rng(3)
    bits = rng.integers(0, 2**63, size=200000, dtype=np.uint64) | (rng.integers(0, 2, 200000, dtype=np.uint64) << 63)
    x = bits.view(np.float64)
    x = x[np.isfinite(x)]
    # moderate magnitudes (the solver's range) with random fractions
    y = rng.standard_normal(200000) * 10.0 ** rng.integers(-30, 30, 200000)
    # exact halfway points between neighbouring floats, and just off them
    f = rng.standard_normal(50000).astype(np.float32)
    g = np.nextafter(f, np.float32(np.inf))
    mid = (f.astype(np.float64) + g.astype(np.float64)) / 2
    near = np.concatenate([mid, np.nextafter(mid, np.inf), np.nextafter(mid, -np.inf)])
    fmax = np.float64(np.finfo(np.float32).max)
    edge = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, fmax, np.nextafter(fmax, np.inf), 2 * fmax, -2 * fmax,
                     1e-38, 1e-40, 1e-45, 7e-46, 1.4e-45, 1e-300, -1e-300, 1.0, -1.0, 0.5,
                     np.float64(np.float32(1.0)) * (1 + 2**-24), 1 - 2**-25, 1 - 2**-26])
    return np.concatenate([x, y, near, edge])


def test_f64_to_f32_bitwise():
    x = torch.from_numpy(_doubles()).cuda()
    got = torch.empty(x.numel(), dtype=torch.float32, device="cuda")
    P.sem_convert(x, got)
    want = x.float()
    torch.cuda.synchronize()
    assert torch.equal(got.view(torch.int32), want.view(torch.int32))


def test_f32_to_f64_bitwise():
    rng = np.random.default_rng(4)
    bits = rng.integers(0, 2**32, size=300000, dtype=np.uint64).astype(np.uint32)
    x = torch.from_numpy(bits.view(np.float32)).cuda()
    got = torch.empty(x.numel(), dtype=torch.float64, device="cuda")
    P.sem_convert(x, got)
    want = x.double()
    torch.cuda.synchronize()
    assert torch.equal(got.view(torch.int64), want.view(torch.int64))
