"""GPU building blocks against the oracle, through the C ABI's kernel-level
entry points: Philox words (bit-exact), Planck group fractions and their
T-derivative (series on the GPU vs quadrature in the oracle), the
time-integrated coefficients, and the linear-frequency sampler (closed-form
root on the GPU vs bisection on the CDF in the oracle)."""
import numpy as np
import pytest

import oracle as O
from paper_2312_16981_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2312_16981_gb300 import binding
    binding.load()
    return binding


def test_philox_bit_exact(B):
    rng = np.random.Generator(np.random.Philox(11))
    ctr = rng.integers(0, 2 ** 32, size=(4099, 4), dtype=np.uint64)
    keys = [(0, 0), (0xDEADBEEF, 0x12345678), (0xFFFFFFFF, 1)]
    for k0, k1 in keys:
        got = B.philox(torch.from_numpy(ctr.astype(np.int64)).to(torch.int32).cuda(), k0, k1).cpu().numpy()
        for i in range(0, len(ctr), 37):
            want = O.philox(ctr[i], (k0, k1))
            np.testing.assert_array_equal(got[i].astype(np.uint32), want)


def test_planck_fractions_match_quadrature(B):
    edges = np.concatenate([I.log_groups(30, 1e-3, 10.0)])
    Ts = np.geomspace(1e-4, 20.0, 61)
    b, d = B.planck(torch.tensor(Ts).cuda(), torch.tensor(edges).cuda())
    b, d = b.cpu().numpy(), d.cpu().numpy()
    worst_b = worst_d = 0.0
    for i, T in enumerate(Ts):
        for g in range(30):
            x1, x2 = edges[g] / T, edges[g + 1] / T
            wb = O.planck_integral(x1, x2)
            wd = O.planck_dintegral(x1, x2)
            if wb > 1e-300:
                worst_b = max(worst_b, abs(b[i, g] - wb) / wb)
            else:
                assert b[i, g] < 1e-290
            if wd > 1e-300:
                worst_d = max(worst_d, abs(d[i, g] - wd) / wd)
    assert worst_b < 2e-13, worst_b
    assert worst_d < 2e-12, worst_d


def test_coefficients_match_oracle(B):
    xs = np.concatenate([np.geomspace(1e-10, 1e4, 400), [0.999999, 1.0, 1.000001]])
    got = B.coefs(torch.tensor(xs).cuda()).cpu().numpy()
    for i, x in enumerate(xs):
        want = O.coefs(x)
        for k in range(4):
            assert abs(got[i, k] - want[k]) <= 1e-13 * abs(want[k]) + 1e-300, (x, k, got[i, k], want[k])


@pytest.mark.parametrize("nlo,nhi,T", [(0.1, 0.13, 1.0), (1.0, 1.36, 0.3), (2.0, 2.7, 0.05),
                                       (5.0, 6.8, 1.0), (0.2, 0.9, 2.0), (9.0, 10.0, 1e-3)])
def test_sampler_matches_bisection(B, nlo, nhi, T):
    rng = np.random.Generator(np.random.Philox(5))
    eta = np.concatenate([rng.random(2000), [1e-12, 0.5, 1 - 1e-12]])
    nu = B.sample_nu(torch.tensor(eta).cuda(), nlo, nhi, T).cpu().numpy()
    for e, v in zip(eta[::7], nu[::7]):
        want = O.sample_nu(nlo, nhi, T, e)
        # the inverse is ill-conditioned only where the clamped density vanishes
        assert abs(v - want) <= 1e-12 * nhi + 2e-8 * (nhi - nlo) * (e < 1e-6 or e > 1 - 1e-6)


@pytest.mark.parametrize("n", [0, 1, 31, 4095, 4096, 4097, 100_003, 1 << 24])
def test_exclusive_scan_bit_exact(B, n):
    rng = np.random.Generator(np.random.Philox(n + 1))
    hi = max(1, min(1 << 12, (1 << 32) // max(n, 1) - 1))
    counts = rng.integers(0, hi, size=n, dtype=np.int64)
    counts[rng.random(n) < 0.3] = 0          # empty bins, as in thick cells
    got = B.exclusive_scan(torch.from_numpy(counts).to(torch.int32).cuda()).cpu().numpy()
    want = np.concatenate([[0], np.cumsum(counts)])
    np.testing.assert_array_equal(got, want)


def test_exclusive_scan_rejects_small_scratch(B):
    import ctypes
    c = torch.zeros(10000, dtype=torch.int32, device="cuda")
    out = torch.zeros(10001, dtype=torch.int32, device="cuda")
    scratch = torch.zeros(4, dtype=torch.uint8, device="cuda")
    code = B.load().ugkwp_exclusive_scan(ctypes.c_void_p(c.data_ptr()), 10000, ctypes.c_void_p(out.data_ptr()),
                                         ctypes.c_void_p(scratch.data_ptr()), 4, None)
    assert code == -7
