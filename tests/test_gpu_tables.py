"""GPU FP64 table generation (trapezoid rule for the Bessel integrals, tanh-sinh
over xi) against the oracle's tables (adaptive Gauss-Legendre), the table file
round trip, and the checks on a damaged file."""
import os

import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    from paper_2110_00256_gb300 import api as a
    return a


def _params(api, ot):
    p = ot.params
    return api.table_params(qs_chi_min=p["qs_chi_min"], qs_chi_max=p["qs_chi_max"], qs_n_chi=p["qs_n_chi"],
                            qs_n_xi=p["qs_n_xi"], qs_xi_min=p["qs_xi_min"], bw_chi_min=p["bw_chi_min"],
                            bw_chi_max=p["bw_chi_max"], bw_n_chi=p["bw_n_chi"], bw_n_xi=p["bw_n_xi"])


@pytest.mark.parametrize("n", [64, 256])
def test_generated_tables_match_oracle(api, n, oracle_tables_256):
    ot = oracle_tables_256 if n == 256 else oracle.tables(qs_n_chi=n, qs_n_xi=n, bw_n_chi=n, bw_n_xi=n)
    t = api.qed_tables_generate(_params(api, ot))
    g = api.qed_tables_copy_to_host(t)
    # 1-D tables: ln G, ln T (absolute in the log = relative in the value)
    assert np.max(np.abs(g["qs_lnG"] - ot.qs_lnG)) < 1e-10
    assert np.max(np.abs(g["bw_lnT"] - ot.bw_lnT)) < 1e-10
    # QS ln P on the log grid
    assert np.max(np.abs(g["qs_lnP"] - ot.qs_lnP)) < 1e-10
    assert np.all(g["qs_lnP"][:, -1] == 0.0)
    # BW P on [0, 1/2]: relative where P is representable, absolute where it underflows
    d = np.abs(g["bw_P"] - ot.bw_P)
    assert np.all(d <= 1e-10 * ot.bw_P + 1e-15)
    assert np.all(g["bw_P"][:, 0] == 0.0) and np.all(g["bw_P"][:, -1] == 0.5)
    assert np.all(np.diff(g["qs_lnP"], axis=1) >= 0) and np.all(np.diff(g["bw_P"], axis=1) >= 0)


def test_generated_tables_are_reproducible(api):
    p = api.table_params(qs_n_chi=32, qs_n_xi=48, bw_n_chi=40, bw_n_xi=24)
    a = api.qed_tables_copy_to_host(api.qed_tables_generate(p))
    b = api.qed_tables_copy_to_host(api.qed_tables_generate(p))
    for k in a:
        assert np.array_equal(a[k], b[k]), k


def test_create_copy_save_load_round_trip(api, tmp_path, oracle_tables_small):
    ot = oracle_tables_small
    t = api.qed_tables_create(_params(api, ot), ot.qs_lnG, ot.qs_lnP, ot.bw_lnT, ot.bw_P)
    h = api.qed_tables_copy_to_host(t)
    for k in ("qs_lnG", "qs_lnP", "bw_lnT", "bw_P"):
        assert np.array_equal(h[k], getattr(ot, k))
    path = str(tmp_path / "tables.qed")
    api.qed_tables_save(t, path)
    t2 = api.qed_tables_load(path)
    h2 = api.qed_tables_copy_to_host(t2)
    for k in h:
        assert np.array_equal(h[k], h2[k])
    p2 = t2.params
    assert p2.qs.n_chi == ot.params["qs_n_chi"] and p2.bw.chi_min == ot.params["bw_chi_min"]
    # a flipped byte in the body fails the checksum; a truncated file fails the size check
    raw = bytearray(open(path, "rb").read())
    raw[len(raw) // 2] ^= 0x40
    bad = str(tmp_path / "bad.qed")
    open(bad, "wb").write(bytes(raw))
    with pytest.raises(api.QedError) as e:
        api.qed_tables_load(bad)
    assert "QED_ERR_IO" in str(e.value)
    open(bad, "wb").write(bytes(raw[:100]))
    with pytest.raises(api.QedError):
        api.qed_tables_load(bad)


def test_generation_rejects_underflowing_range(api):
    # a BW table starting at chi_gamma = 1e-4 has T ~ exp(-26667): ln T is not finite in FP64
    p = api.table_params(qs_n_chi=8, qs_n_xi=8, bw_chi_min=1e-4, bw_n_chi=8, bw_n_xi=8)
    with pytest.raises(api.QedError) as e:
        api.qed_tables_generate(p)
    assert "QED_ERR_NUMERIC" in str(e.value)
