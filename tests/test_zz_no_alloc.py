"""qed_substep_noalloc: the substep for callers that cannot allocate device
memory (their GPU memory belongs to their own pool allocator, or they must not
trigger the device synchronisation of cudaMalloc / cudaFree mid-step).  It keeps
its firing lists in an array compiled into the library instead of taking them
from the caller.  This file is collected last on purpose.

Checked through the C ABI: two consecutive substeps on identical inputs give
the same particles as qed_substep with caller-allocated firing lists, in FP32
and FP64; after a first call, further calls leave the device's free memory and
torch's reserved memory unchanged; and capacities beyond the built-in limit
are rejected before any work is enqueued."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SPECIES = ("electrons", "positrons", "photons")


@pytest.fixture(scope="module")
def api():
    from paper_2110_00256_gb300 import api as a
    return a


@pytest.fixture(scope="module")
def tables(api):
    return api.qed_tables_generate(api.table_params(qs_n_chi=64, qs_n_xi=64, bw_n_chi=64, bw_n_xi=64))


def _inputs(n):
    from paper_2110_00256_gb300 import workloads
    d = {"electrons": workloads.paper_benchmark(n, 101, 0),
         "positrons": workloads.paper_benchmark(n // 4, 102, 10 ** 12),
         "photons": workloads.paper_benchmark(n, 103, 2 * 10 ** 12)}
    for v in d.values():
        v["tau"] *= 3e-4  # a few percent of the particles fire in the first step
    return d


def _buffers(api, host, prec):
    caps = {"electrons": 200_000, "positrons": 100_000, "photons": 300_000}
    return {k: api.SpeciesBuffers(caps[k], prec).set(host[k]) for k in SPECIES}


def _sorted(b):
    h = b.to_host()
    o = np.argsort(h["id"], kind="stable")
    return {k: v[o] for k, v in h.items()}


@pytest.mark.parametrize("prec_name,rtol", [("f32", 1e-5), ("f64", 1e-12)])
def test_noalloc_matches_allocated_substep_twice(api, tables, prec_name, rtol):
    prec = api.QED_F32 if prec_name == "f32" else api.QED_F64
    host = _inputs(100_000)
    ref = _buffers(api, host, prec)
    new = _buffers(api, host, prec)
    fire = [api.FireBuffers(ref[k].capacity) for k in SPECIES]
    s_ref, s_new = api.Stats(), api.Stats()
    for step in (0, 1):
        api.qed_substep(tables, ref["electrons"], ref["positrons"], ref["photons"], 10.0, 17, step, fire,
                        stats=s_ref)
        api.qed_substep_noalloc(tables, new["electrons"], new["positrons"], new["photons"], 10.0, 17, step,
                                stats=s_new)
        torch.cuda.synchronize()
        assert s_ref.as_dict() == s_new.as_dict()
        assert s_new.as_dict()["qs_events"] > 0 and s_new.as_dict()["pairs"] > 0
        for k in SPECIES:
            a, b = _sorted(ref[k]), _sorted(new[k])
            assert np.array_equal(a["id"], b["id"]), (step, k)
            for c in ("px", "py", "pz", "ex", "ey", "ez", "bx", "by", "bz", "tau", "tau_c", "weight"):
                x, y = a[c].astype(np.float64), b[c].astype(np.float64)
                fin = np.isfinite(x)
                assert np.array_equal(fin, np.isfinite(y)), (step, k, c)
                assert np.allclose(y[fin], x[fin], rtol=rtol, atol=0), (step, k, c)


def test_noalloc_allocates_nothing(api, tables):
    host = _inputs(50_000)
    bufs = _buffers(api, host, api.QED_F32)
    stats = api.Stats()
    api.qed_substep_noalloc(tables, bufs["electrons"], bufs["positrons"], bufs["photons"], 10.0, 3, 0, stats=stats)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    reserved0 = torch.cuda.memory_reserved()
    for step in (1, 2):
        api.qed_substep_noalloc(tables, bufs["electrons"], bufs["positrons"], bufs["photons"], 10.0, 3, step,
                                stats=stats)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0 and torch.cuda.memory_reserved() == reserved0
    assert stats.as_dict()["qs_events"] > 0


def test_noalloc_rejects_capacities_beyond_its_limit(api, tables):
    from paper_2110_00256_gb300._lib import QED_NOALLOC_MAX_PARTICLES, QedError
    big = api.SpeciesBuffers(QED_NOALLOC_MAX_PARTICLES // 2 + 1, api.QED_F32)
    small = api.SpeciesBuffers(16, api.QED_F32)
    with pytest.raises(QedError) as e:
        api.qed_substep_noalloc(tables, big, small, big, 1.0, 0, 0)
    assert "QED_ERR_INVALID_ARG" in str(e.value) and "capacities" in str(e.value)
    # one capacity beyond the limit on its own is refused before any sum is formed
    huge = api.SpeciesBuffers(16, api.QED_F32)
    huge.capacity = 2 ** 62  # (never dereferenced: the call is refused first)
    with pytest.raises(QedError) as e:
        api.qed_substep_noalloc(tables, huge, small, huge, 1.0, 0, 0)
    assert "QED_ERR_INVALID_ARG" in str(e.value)
