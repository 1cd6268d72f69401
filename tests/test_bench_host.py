"""Host-side pieces of bench.py that shape its inputs: the numpy chi used to
rescale the fields of the 1000-step QS + BW workload is the §2 definition (the
oracle's chi, particle by particle), so that after rescaling chi follows the
workload's log-uniform target; the headline's configuration is the same in
both arms."""
import numpy as np

import bench
import oracle
from paper_2110_00256_gb300 import workloads


def test_input_chi_is_the_oracles_chi():
    d = workloads.gaussian_fields(200, 5, 1e-3, 1e2)
    for photon in (False, True):
        chi = bench.chi_for_inputs(d, photon)
        f = oracle.chi_photon if photon else oracle.chi_lepton
        for i in range(0, 200, 7):
            p = (d["px"][i], d["py"][i], d["pz"][i])
            E = (d["ex"][i], d["ey"][i], d["ez"][i])
            B = (d["bx"][i], d["by"][i], d["bz"][i])
            ref = f(p, E, B)
            S = np.sqrt(1 + np.dot(p, p)) * np.linalg.norm(E) + np.linalg.norm(p) * np.linalg.norm(B)
            assert abs(chi[i] - ref) <= 1e-12 * S, (photon, i)


def test_rescaled_chi_follows_the_target():
    d = workloads.gaussian_fields(2000, 9, 1e-3, 1e2)
    for photon in (False, True):
        r = workloads.rescale_fields(d, bench.chi_for_inputs(d, photon))
        chi = bench.chi_for_inputs(r, photon)
        assert np.allclose(chi, d["chi_target"], rtol=1e-9)
    lo, hi = np.log10(d["chi_target"].min()), np.log10(d["chi_target"].max())
    assert -3.0 <= lo < -2.9 and 1.9 < hi <= 2.0


def test_headline_config_is_shared_by_both_arms():
    a, b = bench.headline_config(50_000_000, 1), bench.headline_config(50_000_000, 1)
    assert a == b and a["particles"] == 100_000_000 and "sample" not in a
