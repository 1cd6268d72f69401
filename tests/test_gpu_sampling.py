"""The inverse-CDF lookups on the GPU (qed_table_sample, the path the event
kernels take) against the oracle's sampler on the same tables (§3.1, §3.2):
FP64 to rounding; FP32 by its backward error in r through the oracle's forward
map.  Draws include the edges of the guide-table bins, the smallest and largest
uniforms and the BW split r = 1/2; chi spans the out-of-table clamps.  At the
largest table size the guided search equals a linear scan of the interpolated
row."""
import numpy as np
import pytest

from helpers import gpu_tables

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    from paper_2110_00256_gb300 import api as a
    return a


@pytest.fixture(scope="module")
def tabs(api, oracle_tables_256):
    return oracle_tables_256, gpu_tables(api, oracle_tables_256)


def _draws(n, seed, chi_lo, chi_hi):
    r = np.random.default_rng(seed)
    u = r.uniform(0, 1, n)
    edges = np.concatenate([np.arange(1, 128) / 128.0, np.arange(1, 64) / 64.0])
    special = np.concatenate([edges, edges * (1 + 1e-12), edges * (1 - 1e-12), [1e-15, 1e-9, 0.5, 1 - 1e-15]])
    u = np.concatenate([u, special])
    u = np.clip(u, 1e-15, 1 - 1e-15)
    chi = np.exp(r.uniform(np.log(chi_lo), np.log(chi_hi), u.size))
    return chi, u


def _gpu(api, t, proc, prec, chi, u):
    c = torch.as_tensor(chi, device="cuda")
    uu = torch.as_tensor(u, device="cuda")
    return api.qed_table_sample(t, proc, prec, c, uu).cpu().numpy()


@pytest.mark.parametrize("proc", [0, 1])
def test_fp64_sampling_matches_oracle(api, tabs, proc):
    ot, t = tabs
    chi, u = _draws(20000, 3 + proc, 1e-4, 1e4)
    got = _gpu(api, t, proc, api.QED_F64, chi, u)
    if proc == 0:
        ref = np.array([ot.qs_sample_xi(c, x) for c, x in zip(chi, u)])
        assert np.allclose(got, ref, rtol=1e-10, atol=0)
    else:
        ref = []
        for c, x in zip(chi, u):
            xs, e = ot.bw_sample_xi(c, x)
            ref.append(xs if e else 1.0 - xs)
        assert np.allclose(got, np.array(ref), rtol=0, atol=1e-12)


@pytest.mark.parametrize("proc", [0, 1])
def test_fp32_sampling_backward_error(api, tabs, proc):
    """the r that the FP32 sample maps back to (oracle forward map at the
    FP32-rounded chi) is the FP32 draw to 1e-5 relative"""
    ot, t = tabs
    chi, u = _draws(20000, 7 + proc, 1e-4, 1e4)
    got = _gpu(api, t, proc, api.QED_F32, chi, u)
    c32 = chi.astype(np.float32).astype(np.float64)
    bad = 0
    for c, x, xi in zip(c32, u, got):
        if proc == 0:
            r = float(np.float32(x)) if np.float32(x) <= x else float(np.nextafter(np.float32(x), np.float32(0)))
            back = ot.qs_table_cdf(c, xi)
        else:
            fold = x if x <= 0.5 else 1.0 - x
            r = float(np.float32(fold)) if np.float32(fold) <= fold else float(np.nextafter(np.float32(fold),
                                                                                             np.float32(0)))
            lep = xi if x <= 0.5 else 1.0 - xi
            back = ot.bw_table_cdf(c, lep)
        bad += abs(back - r) > 1e-5 * r + 1e-12
    assert bad == 0


def test_guided_search_equals_linear_scan_at_max_size(api):
    """1024 x 1024 tables made on the GPU: FP64 samples equal the same
    interpolation evaluated on the host with a linear scan of the row"""
    n = 1024
    t = api.qed_tables_generate(api.table_params(qs_n_chi=n, qs_n_xi=n, bw_n_chi=n, bw_n_xi=n))
    h = api.qed_tables_copy_to_host(t)
    p = t.params
    for proc in (0, 1):
        ax = p.qs if proc == 0 else p.bw
        rows = h["qs_lnP"] if proc == 0 else h["bw_P"]
        rows = rows.reshape(n, n)
        chi, u = _draws(3000, 11 + proc, ax.chi_min, ax.chi_max)
        got = _gpu(api, t, proc, api.QED_F64, chi, u)
        l0, l1 = np.log(ax.chi_min), np.log(ax.chi_max)
        tt = np.clip((np.log(chi) - l0) * ((n - 1) / (l1 - l0)), 0, n - 1)
        k = np.minimum(tt.astype(int), n - 2)
        w = tt - k
        for i in range(chi.size):
            row = rows[k[i]] + w[i] * (rows[k[i] + 1] - rows[k[i]])
            if proc == 0:
                x = np.log(u[i])
                xs = np.log(ax.xi_min) + np.arange(n) * (-np.log(ax.xi_min) / (n - 1))
            else:
                x = u[i] if u[i] <= 0.5 else 1.0 - u[i]
                xs = 0.5 * np.arange(n) / (n - 1)
            m = int(np.searchsorted(row, x, side="right")) - 1
            m = min(max(m, 0), n - 2)
            if row[m + 1] == row[m]:
                v = xs[m]
            else:
                v = xs[m] + (x - row[m]) * (xs[m + 1] - xs[m]) / (row[m + 1] - row[m])
            if proc == 0:
                ref = np.exp(min(v, 0.0))
            else:
                v = min(max(v, 0.0), 0.5)
                ref = v if u[i] <= 0.5 else 1.0 - v
            assert got[i] == pytest.approx(ref, rel=1e-9, abs=1e-13), (proc, i, chi[i], u[i])
