"""Shared helpers of the GPU parity tests: run the CUDA path through the C ABI
and compare it with the FP64 oracle on identical seeded inputs.

Tolerances.  Continuous outputs must agree to 1e-12 (FP64) / 1e-5 (FP32)
relative to the scale of the terms that form them:
  - chi to tol * S with S = gamma |E| + |p| |B| (photons: |p| (|E| + |B|)),
    widened by the FP64 rounding bound of a difference-of-squares evaluation
    (the oracle's, and the GPU's FP64 path), 16 eps S^2 / chi;
  - the optical depth to tol |tau_old| + dt * (the rate change that this chi
    uncertainty produces through the oracle's table lookup, plus tol * rate);
  - a firing decision may differ only where the oracle's new optical depth lies
    within that bound of zero (and, in FP64, within the stated 1e-6 margin);
  - an FP32 inverse-CDF sample is assessed by its backward error: the r that the
    oracle's FP64 table maps to the sampled xi must lie within 1e-5 (relative)
    of the drawn uniform (1e-12 for FP64 samples where chi itself differs, see
    check_substep_by_event).
"""
import numpy as np

import oracle

FIELDS = ("px", "py", "pz", "ex", "ey", "ez", "bx", "by", "bz")
TOL = {"f64": 1e-12, "f32": 1e-5}
MARGIN_F64 = 1e-6
EPS64 = 2.0 ** -53


def gpu_tables(api, ot):
    p = api.table_params(qs_chi_min=ot.params["qs_chi_min"], qs_chi_max=ot.params["qs_chi_max"],
                         qs_n_chi=ot.params["qs_n_chi"], qs_n_xi=ot.params["qs_n_xi"],
                         qs_xi_min=ot.params["qs_xi_min"], bw_chi_min=ot.params["bw_chi_min"],
                         bw_chi_max=ot.params["bw_chi_max"], bw_n_chi=ot.params["bw_n_chi"],
                         bw_n_xi=ot.params["bw_n_xi"])
    return api.qed_tables_create(p, ot.qs_lnG, ot.qs_lnP, ot.bw_lnT, ot.bw_P)


def as_f64(d, dtype):
    """Round the inputs to the working precision, return them as FP64 for the oracle."""
    out = {}
    for k, v in d.items():
        if k == "id":
            out[k] = np.asarray(v, dtype=np.uint64)
        elif k == "chi_target":
            continue
        else:
            out[k] = np.asarray(v, dtype=dtype).astype(np.float64)
    return out


def tau_eff(h, prec_f32):
    """The optical depth the GPU holds: tau - tau_c in FP32 (Kahan pair), tau in FP64."""
    t = h["tau"].astype(np.float64)
    if prec_f32:
        t = t - h["tau_c"].astype(np.float64)
    return t


def _norm(d, a, b, c):
    return np.sqrt(d[a] ** 2 + d[b] ** 2 + d[c] ** 2)


def energy_of(proc, d):
    p2 = d["px"] ** 2 + d["py"] ** 2 + d["pz"] ** 2
    return np.sqrt(1.0 + p2) if proc == 0 else np.sqrt(p2)


def chi_scale(proc, d):
    E = _norm(d, "ex", "ey", "ez")
    B = _norm(d, "bx", "by", "bz")
    return energy_of(proc, d) * E + _norm(d, "px", "py", "pz") * B


def tau_bound(ot, proc, d, chi, rate, dt, tol):
    """Allowed |tau_gpu - tau_oracle| after one evolution step (module docstring)."""
    S = chi_scale(proc, d)
    dchi = tol * S + 16 * EPS64 * S * S / np.maximum(chi, 1e-300)
    en = energy_of(proc, d)
    r_hi = ot.rates(proc, chi + dchi, en)
    r_lo = ot.rates(proc, np.maximum(chi - dchi, 0.0), en)
    drate = np.maximum(np.abs(r_hi - rate), np.abs(r_lo - rate)) + tol * rate
    return tol * np.abs(d["tau"] - d.get("tau_c", 0.0)) + dt * drate + 1e-300


def compare_evolve(name, got_tau, got_fire_idx, got_fire_chi, inp, proc, ot, dt, tol, f64):
    """Optical depths and firing sets of one species against the oracle.
    Returns the indices whose decision differs (all within the bound)."""
    tau_new, chi, rate, fire = oracle.evolve(proc, ot, inp, dt)
    bound = tau_bound(ot, proc, inp, chi, rate, dt, tol)
    fin = np.isfinite(tau_new)
    assert np.array_equal(np.isfinite(got_tau), fin), f"{name}: finite mask"
    err = np.abs(got_tau - tau_new)
    bad = fin & (err > bound)
    assert not bad.any(), f"{name}: {bad.sum()} optical depths outside the bound; worst ratio " \
                          f"{np.max(err[fin] / bound[fin]):.3e}"
    gf = np.zeros(tau_new.shape[0], dtype=bool)
    gf[got_fire_idx] = True
    assert len(np.unique(got_fire_idx)) == len(got_fire_idx), f"{name}: duplicate firing entries"
    diff = np.nonzero(gf != fire)[0]
    assert np.all(np.abs(tau_new[diff]) <= bound[diff]), f"{name}: decisions differ outside the error bound"
    if f64:
        scale = np.abs(inp["tau"]) + rate * dt
        assert np.all(np.abs(tau_new[diff]) < MARGIN_F64 * scale[diff]), f"{name}: outside the 1e-6 margin"
    if len(got_fire_idx):
        S = chi_scale(proc, {k: v[got_fire_idx] for k, v in inp.items()})
        c_ref = chi[got_fire_idx]
        dchi = tol * S + 16 * EPS64 * S * S / np.maximum(c_ref, 1e-300)
        assert np.all(np.abs(got_fire_chi - c_ref) <= dchi), f"{name}: chi in the firing list"
    return diff


def sort_by_id(d):
    o = np.argsort(d["id"], kind="stable")
    return {k: v[o] for k, v in d.items()}


def check_substep_by_event(ot, host, got, fire_lists, dt, seed, step, fp64=False):
    """Element-wise check of one substep, event by event (see module docstring).
    host: pre-step state as FP64 (from the inputs in the working precision);
    got: GPU state after; fire_lists: species -> (indices, chi) of the GPU
    firing lists.  The sample of a firing particle is assessed at the chi the
    GPU evaluated (its own error is bounded separately, against the oracle's
    chi) by its backward error.  FP64 (fp64=True) takes the FP64 tolerances:
    used where the chi of many events differ from the oracle's by the FP64
    cancellation bound of a small chi, which a sampled xi would inherit."""
    tol = TOL["f64"] if fp64 else TOL["f32"]
    rtol_r = 1e-12 if fp64 else 1e-5          # backward error of a sample
    rtol_e = 1e-12 if fp64 else 4e-7          # energy and direction of the products
    procs = {"electrons": 0, "positrons": 0, "photons": 1}
    gpu = {k: {kk: v for kk, v in got[k].items()} for k in got}
    by_id = {k: {int(i): j for j, i in enumerate(gpu[k]["id"])} for k in gpu}
    report = {"events": 0, "worst_r": 0.0, "decision_diffs": 0}
    for name, proc in procs.items():
        h = host[name]
        n = len(h["px"])
        if n == 0:
            continue
        tau_new, chi, rate, fire = oracle.evolve(proc, ot, h, dt)
        bound = tau_bound(ot, proc, h, chi, rate, dt, tol)
        g = gpu[name]
        idx = np.array([by_id[name][int(i)] for i in h["id"]])
        gt = tau_eff({k: v[idx] for k, v in g.items()}, not fp64)
        gp = {c: g[c][idx].astype(np.float64) for c in FIELDS}
        gw = g["weight"][idx].astype(np.float64)
        # which ones fired on the GPU: leptons have a reset tau and a photon child;
        # photons are removed (or reset when below the pair threshold)
        if proc == 0:
            moved = ~((gp["px"] == h["px"]) & (gp["py"] == h["py"]) & (gp["pz"] == h["pz"]))
            cid = np.array([oracle.child_ids(seed, int(i), step)[0] for i in h["id"]], dtype=np.uint64)
            has_child = np.array([int(c) in by_id["photons"] for c in cid])
            gfire = has_child | moved
        else:
            gfire = (gw == 0) | (~np.isfinite(gt))
        diff = np.nonzero(gfire != fire)[0]
        assert np.all(np.abs(tau_new[diff]) <= bound[diff]), f"{name}: decision outside the bound"
        report["decision_diffs"] += len(diff)
        same = gfire == fire
        quiet = same & ~fire
        err = np.abs(gt[quiet] - tau_new[quiet])
        assert np.all(err <= bound[quiet]), f"{name}: optical depth outside the bound"
        for c in FIELDS:
            assert np.array_equal(gp[c][quiet], h[c][quiet]), f"{name}: {c} changed without an event"
        ev = np.nonzero(same & fire)[0]
        report["events"] += len(ev)
        fidx, fchi = fire_lists[name]
        chi_gpu = dict(zip(fidx.tolist(), fchi.tolist()))
        S = chi_scale(proc, h)
        dchi = tol * S + 16 * EPS64 * S * S / np.maximum(chi, 1e-300)
        for j in ev:
            assert abs(chi_gpu[int(j)] - chi[j]) <= dchi[j], (name, j)
        for j in ev:
            pid = int(h["id"][j])
            r = oracle.uniform(seed, pid, step, oracle.PURPOSE_SAMPLE)
            pm = np.sqrt(h["px"][j] ** 2 + h["py"][j] ** 2 + h["pz"][j] ** 2)
            nvec = np.array([h["px"][j], h["py"][j], h["pz"][j]]) / pm
            if proc == 0:
                gam = np.sqrt(1.0 + pm * pm)
                c0, _ = oracle.child_ids(seed, pid, step)
                ph = gpu["photons"]
                k = by_id["photons"][c0]
                pg = np.array([ph["px"][k], ph["py"][k], ph["pz"][k]], dtype=np.float64)
                gg = np.linalg.norm(pg)
                xi = gg / (gam - 1.0)
                rr = ot.qs_table_cdf(chi_gpu[int(j)], xi)
                report["worst_r"] = max(report["worst_r"], abs(rr - r) / r)
                assert abs(rr - r) <= rtol_r * r, (name, pid, r, rr)
                # recoil: energy conserved to the working precision's rounding, direction kept
                pl = np.array([gp["px"][j], gp["py"][j], gp["pz"][j]])
                gl = np.sqrt(1.0 + pl @ pl)
                assert abs(gl + gg - gam) <= rtol_e * gam, (name, pid)
                assert np.linalg.norm(np.cross(pl, nvec)) <= rtol_e * (np.linalg.norm(pl) + 1.0)
                assert np.linalg.norm(np.cross(pg, nvec)) <= rtol_e * (gg + 1e-30)
                want_tau = oracle.tau_draw(seed, pid, step, oracle.PURPOSE_TAU_RESET)
                assert abs(gt[j] - want_tau) <= 1e-12 * want_tau
                assert abs(tau_eff({kk: v[k:k + 1] for kk, v in ph.items()}, not fp64)[0]
                           - oracle.tau_draw(seed, c0, step, oracle.PURPOSE_TAU_INIT)) <= 1e-12 * 40
                for c in ("ex", "ey", "ez", "bx", "by", "bz", "weight"):
                    assert float(ph[c][k]) == float(h[c][j])
            else:
                if pm <= 2.0:
                    continue
                ce, cp = oracle.child_ids(seed, pid, step)
                e, q = gpu["electrons"], gpu["positrons"]
                ke, kq = by_id["electrons"][ce], by_id["positrons"][cp]
                pe = np.array([e["px"][ke], e["py"][ke], e["pz"][ke]], dtype=np.float64)
                pq = np.array([q["px"][kq], q["py"][kq], q["pz"][kq]], dtype=np.float64)
                ge, gq = np.sqrt(1 + pe @ pe), np.sqrt(1 + pq @ pq)
                assert abs(ge + gq - pm) <= rtol_e * pm, (name, pid)
                km = (pe @ pe) / (ge + 1.0)  # kinetic energy, accurate for small momenta
                kp = (pq @ pq) / (gq + 1.0)
                electron = r <= 0.5
                xs = (km if electron else kp) / (pm - 2.0)
                rs = r if electron else 1.0 - r
                rr = ot.bw_table_cdf(chi_gpu[int(j)], xs)
                report["worst_r"] = max(report["worst_r"], abs(rr - rs) / rs)
                assert abs(rr - rs) <= rtol_r * rs + 1e-12, (name, pid, rs, rr)
                assert gw[j] == 0 and np.isinf(gt[j])
    return report


def margin_ids(ot, host64, dt, tol, seed, step, cuts=(0.0, 0.0)):
    """ids of particles whose decision lies within the error bound (of the
    firing test or of a chi cut-off), and their children."""
    out = set()
    for k, proc in (("electrons", 0), ("positrons", 0), ("photons", 1)):
        tn, chi, rate, f = oracle.evolve(proc, ot, host64[k], dt, cuts[proc])
        b = tau_bound(ot, proc, host64[k], chi, rate, dt, tol)
        near_cut = np.abs(chi - cuts[proc]) <= 1e-9 * cuts[proc]
        # (removed photons, tau = +inf, take no decision)
        for pid in host64[k]["id"][np.isfinite(tn) & ((np.abs(tn) <= b) | near_cut)].tolist():
            out.add(pid)
            out |= set(oracle.child_ids(seed, pid, step))
    return out


def compare_states(got, ref, prec_f32, tol, exclude=frozenset()):
    worst = {}
    for k in ("electrons", "positrons", "photons"):
        g, r = sort_by_id(got[k]), sort_by_id({kk: ref[k][kk] for kk in got[k]})
        if exclude:
            keep_g = ~np.isin(g["id"], list(exclude))
            keep_r = ~np.isin(r["id"], list(exclude))
            g = {kk: v[keep_g] for kk, v in g.items()}
            r = {kk: v[keep_r] for kk, v in r.items()}
        assert np.array_equal(g["id"], r["id"]), f"{k}: id sets differ ({len(g['id'])} vs {len(r['id'])})"
        gt = tau_eff(g, prec_f32)
        fin = np.isfinite(r["tau"])
        assert np.array_equal(np.isfinite(gt), fin), f"{k}: removed-particle mask"
        pm = np.sqrt(r["px"] ** 2 + r["py"] ** 2 + r["pz"] ** 2)
        e = 0.0
        for c in ("px", "py", "pz"):
            e = max(e, float(np.max(np.abs(g[c] - r[c]) / np.maximum(pm, 1e-300), initial=0)))
        et = float(np.max(np.abs(gt[fin] - r["tau"][fin]) / np.maximum(np.abs(r["tau"][fin]), 1.0), initial=0))
        for c in ("ex", "ey", "ez", "bx", "by", "bz", "weight"):
            assert np.array_equal(g[c].astype(np.float64), r[c]), f"{k}: {c} copied exactly"
        worst[k] = (e, et)
        assert e <= tol, f"{k}: momentum rel err {e:.3e}"
        assert et <= tol, f"{k}: tau err {et:.3e}"
    return worst
