"""The FP64 logarithm and exponential of the rate lookups (Tang's table-driven
forms, csrc/fp64_math.cuh) against the host's libm (numpy) and the CUDA
library on the same inputs, over the whole double range: the exponential within
2 ulp, the logarithm within 2 ulp plus 2^-57 absolute; the special values
(0, subnormals, the overflow and underflow edges, inf, NaN) as IEEE defines."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    from paper_2110_00256_gb300 import api as a
    return a


def _ulps(a, ref):
    with np.errstate(invalid="ignore"):
        return np.where(a == ref, 0.0, np.abs(a - ref) / np.spacing(np.abs(ref)))


def _run(api, x):
    r = api.qed_probe_fp64_logexp(torch.tensor(x, dtype=torch.float64, device="cuda"))
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in r.items()}


def test_exp_within_two_ulp(api):
    rng = np.random.default_rng(5)
    x = np.concatenate([rng.uniform(-745.2, 709.8, 400_000), rng.uniform(-1, 1, 200_000),
                        rng.uniform(-1e-3, 1e-3, 100_000), rng.uniform(-60, 60, 200_000),
                        np.linspace(707.9, 709.78, 5000), np.linspace(-708.1, -745.1, 5000),
                        [0.0, -0.0, 1e-300, -1e-300, 708.0, -708.0, 709.78, -745.13]])
    with np.errstate(over="ignore", under="ignore"):
        ref = np.exp(x)
    r = _run(api, x)
    for name in ("exp", "exp_lib"):
        u = _ulps(r[name], ref)
        print(f"{name}: max {u.max():.2f} ulp, mean {u.mean():.3f}")
        assert u.max() <= 2.0, (name, x[np.argmax(u)], u.max())


def test_log_within_two_ulp_and_absolute(api):
    rng = np.random.default_rng(6)
    e = rng.uniform(-1074, 1024, 400_000)
    x = np.concatenate([np.exp2(e) * rng.uniform(1, 2, e.size), rng.uniform(0.5, 2, 200_000),
                        1 + rng.uniform(-1e-3, 1e-3, 100_000), rng.uniform(1e-3, 1e3, 200_000),
                        [5e-324, 1e-310, 2.2250738585072014e-308, 1.0, 2.0, 0.5, 1.7976931348623157e308]])
    x = x[np.isfinite(x) & (x > 0)]
    ref = np.log(x)
    r = _run(api, x)
    for name in ("log", "log_lib"):
        err = np.abs(r[name] - ref)
        bound = 2 * np.spacing(np.abs(ref)) + 2.0 ** -57
        print(f"{name}: max err / bound {np.max(err / bound):.3f}, max ulp away from 1: "
              f"{_ulps(r[name], ref)[np.abs(ref) > 0.05].max():.2f}")
        assert np.all(err <= bound), (name, x[np.argmax(err / bound)])
    assert np.all(_ulps(r["log"], ref)[np.abs(ref) > 0.05] <= 2.0)


def test_special_values(api):
    inf, nan = np.inf, np.nan
    x = np.array([0.0, -0.0, -1.0, inf, -inf, nan, 710.0, -746.0, 1e6, -1e6, 5e-324])
    r = _run(api, x)
    lg, ex = r["log"], r["exp"]
    assert lg[0] == -inf and lg[1] == -inf and np.isnan(lg[2]) and lg[3] == inf and np.isnan(lg[4])
    assert np.isnan(lg[5]) and lg[10] == pytest.approx(np.log(5e-324), rel=1e-15)
    assert ex[0] == 1.0 and ex[1] == 1.0 and ex[3] == inf and ex[4] == 0.0 and np.isnan(ex[5])
    assert ex[6] == inf and ex[7] == 0.0 and ex[8] == inf and ex[9] == 0.0
    for k in ("log", "exp"):
        lib = r[k + "_lib"]
        same = (r[k] == lib) | (np.isnan(r[k]) & np.isnan(lib))
        assert np.all(same[:10]), (k, r[k], lib)
