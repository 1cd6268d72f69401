"""Every entry point on empty inputs: nothing runs, nothing is appended,
statistics stay zero, and the calls return QED_OK (FP32 and FP64)."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    from paper_2110_00256_gb300 import api as a
    return a


@pytest.fixture(scope="module")
def tables(api):
    return api.qed_tables_generate(api.table_params(qs_n_chi=64, qs_n_xi=64, bw_n_chi=64, bw_n_xi=64))


@pytest.mark.parametrize("prec_name", ["f32", "f64"])
def test_empty_everything(api, tables, prec_name):
    prec = api.QED_F32 if prec_name == "f32" else api.QED_F64
    sp = {k: api.SpeciesBuffers(64, prec, positions=True) for k in ("electrons", "positrons", "photons")}
    fire = [api.FireBuffers(64) for _ in range(3)]
    st = api.Stats()
    api.qed_init_optical_depth(sp["electrons"], 1)
    api.qed_evolve_optical_depth(tables, 0, sp["electrons"], 10.0, fire[0], st)
    api.qed_substep(tables, sp["electrons"], sp["positrons"], sp["photons"], 10.0, 1, 0, fire, stats=st)
    api.qed_substep_noalloc(tables, sp["electrons"], sp["positrons"], sp["photons"], 10.0, 1, 0, stats=st)
    w = api.plane_wave(1e-4, 3e-6)
    for k, q in (("electrons", -1.0), ("positrons", 1.0), ("photons", 0.0)):
        api.qed_push_plane_wave(sp[k], q, w, 0.0, 10.0)
        api.qed_push_stored_fields(sp[k], q, 10.0)
    patch = dict(sp, fire=fire)
    b = api.Batch([patch, dict(patch)], prec)
    api.qed_substep_batched(tables, b, 10.0, 1, 0, api.make_opts(stats=st))
    api.qed_push_batched(b, w, 0.0, 10.0, 0)
    api.qed_push_substep_batched(tables, b, w, 0.0, 10.0, 1, 1, api.make_opts(stats=st))
    td = torch.float32 if prec == api.QED_F32 else torch.float64
    cells = {k: torch.empty(0, device="cuda", dtype=td) for k in ("ex", "ey", "ez", "bx", "by", "bz")}
    api.qed_schwinger_pairs(cells, 1.0, 1.0, 1.0, 1, 0, sp["electrons"], sp["positrons"], stats=st)
    e = torch.empty(0, device="cuda", dtype=torch.float64)
    api.qed_table_sample(tables, 0, prec, e, e)
    torch.cuda.synchronize()
    assert all(v == 0 for v in st.as_dict().values())
    assert all(sp[k].n() == 0 for k in sp) and all(f.n() == 0 for f in fire)
