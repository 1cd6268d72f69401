"""Host-side checks of the learned sampler's evaluation helper
(paper_2110_00256_gb300.surrogate.ks_distance, the two-sample Kolmogorov-Smirnov
distance that the bench and the sampler-quality tests report): it equals
scipy's statistic, vanishes for identical samples and is symmetric."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
stats = pytest.importorskip("scipy.stats")


def test_ks_distance_matches_scipy():
    from paper_2110_00256_gb300.surrogate import ks_distance
    rng = np.random.default_rng(3)
    for n, m, shift in ((1000, 1000, 0.0), (2000, 700, 0.1), (500, 1500, 0.5)):
        a = rng.normal(0.0, 1.0, n)
        b = rng.normal(shift, 1.0, m)
        d = ks_distance(torch.tensor(a), torch.tensor(b))
        assert d == pytest.approx(stats.ks_2samp(a, b).statistic, abs=1e-12)
        assert d == pytest.approx(ks_distance(torch.tensor(b), torch.tensor(a)), abs=1e-15)
    x = torch.tensor(rng.uniform(0, 1, 4000))
    assert ks_distance(x, x.clone()) == 0.0
