"""Pins of the oracle's forward maps of the table sampling (§3.1, §3.2).

``qs_table_cdf`` / ``bw_table_cdf`` give the r that the inverse-CDF lookup maps
to a xi: the interpolated row of the 2-D table evaluated at xi.  They are the
checker of every FP32 sampling assertion (backward error) and of the kinetic
reference of the tabulated method, so they are pinned here against things
other than themselves:

* at the grid nodes they return the stored table entries (index arithmetic,
  row/column order);
* between nodes they follow the paper's interpolants: log-log in (chi, xi) for
  QS (§3.2), linear in ln chi and in xi for BW (§3.1): a geometric midpoint in
  xi gives the geometric mean of the two CDF values (QS) and an arithmetic
  midpoint the arithmetic mean (BW);
* they invert the samplers (``qs_sample_xi`` / ``bw_sample_xi``, the paper's
  binary-search-and-interpolate lookup written as a scan): table_cdf(chi,
  sample_xi(chi, r)) == r on stratified r, at and between chi nodes, outside
  the chi range (clamped), at the xi-interval edges, and below P(xi_min) where
  the first QS segment is extrapolated log-log.
"""
import math

import numpy as np
import pytest

import oracle


def _chi_node(t, proc, n):
    p = t.params
    pre = "qs" if proc == 0 else "bw"
    l0, l1, N = math.log(p[pre + "_chi_min"]), math.log(p[pre + "_chi_max"]), p[pre + "_n_chi"]
    return math.exp(l0 + n * (l1 - l0) / (N - 1))


def _qs_xi_node(t, m):
    p = t.params
    lx0, M = math.log(p["qs_xi_min"]), p["qs_n_xi"]
    return math.exp(lx0 + m * (0.0 - lx0) / (M - 1))


def _rows(t, proc):
    p = t.params
    if proc == 0:
        return t.qs_lnP.reshape(p["qs_n_chi"], p["qs_n_xi"])
    return t.bw_P.reshape(p["bw_n_chi"], p["bw_n_xi"])


@pytest.mark.parametrize("n", (0, 7, 31, 62))
def test_qs_forward_map_at_nodes(oracle_tables_small, n):
    t = oracle_tables_small
    rows = _rows(t, 0)
    chi = _chi_node(t, 0, n)
    for m in (0, 1, 17, 40, 62, 63):
        got = t.qs_table_cdf(chi, _qs_xi_node(t, m))
        assert got == pytest.approx(math.exp(rows[n, m]), rel=1e-12), (n, m)


@pytest.mark.parametrize("n", (0, 9, 33, 62))
def test_bw_forward_map_at_nodes(oracle_tables_small, n):
    t = oracle_tables_small
    rows = _rows(t, 1)
    M = t.params["bw_n_xi"]
    chi = _chi_node(t, 1, n)
    for m in (0, 1, 20, 50, M - 1):
        got = t.bw_table_cdf(chi, 0.5 * m / (M - 1))
        assert got == pytest.approx(rows[n, m], rel=1e-12, abs=1e-300), (n, m)


def test_qs_forward_map_is_log_log_between_nodes(oracle_tables_small):
    t = oracle_tables_small
    rows = _rows(t, 0)
    n, m = 20, 45
    # geometric midpoint in xi at a chi node: geometric mean of the two CDF values
    xa, xb = _qs_xi_node(t, m), _qs_xi_node(t, m + 1)
    got = t.qs_table_cdf(_chi_node(t, 0, n), math.sqrt(xa * xb))
    assert got == pytest.approx(math.exp(0.5 * (rows[n, m] + rows[n, m + 1])), rel=1e-12)
    # an arithmetic midpoint would give the arithmetic mean instead: the two differ here
    lin = 0.5 * (math.exp(rows[n, m]) + math.exp(rows[n, m + 1]))
    assert abs(got / lin - 1.0) > 1e-6
    # geometric midpoint in chi at a xi node
    ca, cb = _chi_node(t, 0, n), _chi_node(t, 0, n + 1)
    got = t.qs_table_cdf(math.sqrt(ca * cb), _qs_xi_node(t, m))
    assert got == pytest.approx(math.exp(0.5 * (rows[n, m] + rows[n + 1, m])), rel=1e-12)


def test_bw_forward_map_is_linear_between_nodes(oracle_tables_small):
    t = oracle_tables_small
    rows = _rows(t, 1)
    M = t.params["bw_n_xi"]
    n, m = 40, 30
    x = 0.5 * (m + 0.5) / (M - 1)
    got = t.bw_table_cdf(_chi_node(t, 1, n), x)
    assert got == pytest.approx(0.5 * (rows[n, m] + rows[n, m + 1]), rel=1e-12)
    ca, cb = _chi_node(t, 1, n), _chi_node(t, 1, n + 1)
    got = t.bw_table_cdf(math.sqrt(ca * cb), 0.5 * m / (M - 1))
    assert got == pytest.approx(0.5 * (rows[n, m] + rows[n + 1, m]), rel=1e-12)


def _qs_chis(t):
    return (t.params["qs_chi_min"] * 0.3, _chi_node(t, 0, 5), 0.0371, 1.0, 9.0, _chi_node(t, 0, 40) * 1.0001,
            257.0, t.params["qs_chi_max"] * 4.0)


def _bw_chis(t):
    return (t.params["bw_chi_min"] * 0.5, 0.05, _chi_node(t, 1, 12), 1.0, 13.7, 400.0, t.params["bw_chi_max"] * 2)


@pytest.mark.parametrize("table", ("small", "256"))
def test_qs_forward_map_inverts_the_sampler(oracle_tables_small, oracle_tables_256, table):
    t = oracle_tables_small if table == "small" else oracle_tables_256
    r = np.concatenate([(np.arange(400) + 0.5) / 400, [1e-9, 1e-7, 1e-5, 1e-3, 1 - 1e-6, 1 - 1e-12]])
    for chi in _qs_chis(t):
        lc = math.log(min(max(chi, t.params["qs_chi_min"]), t.params["qs_chi_max"]))
        for v in r:
            xi = t.qs_sample_xi(chi, v)
            assert 0.0 < xi <= 1.0
            if xi == 1.0:  # clamped at the table's last column: r beyond the row's last value
                continue
            back = t.qs_table_cdf(chi, xi)
            assert back == pytest.approx(v, rel=1e-10), (chi, v, xi)
        # the row's own values as r: the sampler returns the xi node (interval edges)
        rows = _rows(t, 0)
        p = t.params
        l0, l1, N = math.log(p["qs_chi_min"]), math.log(p["qs_chi_max"]), p["qs_n_chi"]
        n = min(int((lc - l0) / ((l1 - l0) / (N - 1))), N - 2)
        w = (lc - (l0 + n * (l1 - l0) / (N - 1))) / ((l1 - l0) / (N - 1))
        row = rows[n] + w * (rows[n + 1] - rows[n])
        for m in (3, 100 if p["qs_n_xi"] > 128 else 30, p["qs_n_xi"] - 3):
            if not (row[m - 1] + 1e-9 < row[m] < row[m + 1] - 1e-9):
                # a flat stretch (ln P = 0 to within rounding at small chi): r = exp(ln P_m)
                # does not single out node m after rounding
                continue
            xi = t.qs_sample_xi(chi, math.exp(row[m]))
            assert xi == pytest.approx(_qs_xi_node(t, m), rel=1e-9), (chi, m)


def test_qs_sampler_extrapolates_below_xi_min(oracle_tables_256):
    """r below the row's first value: xi < xi_min on the first segment's
    log-log line (the xi^(1/3) power law of the number spectrum)."""
    t = oracle_tables_256
    chi = 2.0
    p0 = t.qs_table_cdf(chi, t.params["qs_xi_min"])
    for f in (0.5, 1e-3, 1e-6):
        xi = t.qs_sample_xi(chi, p0 * f)
        assert xi < t.params["qs_xi_min"]
        assert t.qs_table_cdf(chi, xi) == pytest.approx(p0 * f, rel=1e-10)
        # slope of the extrapolation ~ 1/3 in log-log
        assert math.log(f) / math.log(xi / t.params["qs_xi_min"]) == pytest.approx(1.0 / 3.0, rel=2e-2)


@pytest.mark.parametrize("table", ("small", "256"))
def test_bw_forward_map_inverts_the_sampler(oracle_tables_small, oracle_tables_256, table):
    t = oracle_tables_small if table == "small" else oracle_tables_256
    r = np.concatenate([(np.arange(400) + 0.5) / 400, [1e-12, 0.5, 0.5 + 1e-12, 1 - 1e-12]])
    for chi in _bw_chis(t):
        for v in r:
            xi, is_el = t.bw_sample_xi(chi, v)
            assert is_el == (v <= 0.5)
            rf = v if v <= 0.5 else 1.0 - v
            if xi == 0.0 or xi == 0.5:
                # a flat end segment (P = 0 below the first nonzero column, or the
                # row's value 1/2 reached): nothing to invert
                continue
            back = t.bw_table_cdf(chi, xi)
            assert back == pytest.approx(rf, rel=1e-10, abs=1e-15), (chi, v, xi)


def test_forward_map_clamps_chi_outside_the_table(oracle_tables_small):
    t = oracle_tables_small
    p = t.params
    for xi in (1e-6, 0.3, 0.97):
        assert t.qs_table_cdf(p["qs_chi_min"] * 1e-3, xi) == t.qs_table_cdf(p["qs_chi_min"], xi)
        assert t.qs_table_cdf(p["qs_chi_max"] * 1e3, xi) == t.qs_table_cdf(p["qs_chi_max"], xi)
    for xi in (0.01, 0.2, 0.49):
        assert t.bw_table_cdf(p["bw_chi_min"] * 1e-2, xi) == t.bw_table_cdf(p["bw_chi_min"], xi)
        assert t.bw_table_cdf(p["bw_chi_max"] * 1e2, xi) == t.bw_table_cdf(p["bw_chi_max"], xi)
