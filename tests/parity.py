"""Comparison of the CUDA chain's output with the CPU oracle (test infrastructure).

Objects are compared as canonical sets: every object is identified by its tuple of input hit
indices (seed objects also by the seed index). With D the oracle's definite objects (every cut clear
of its threshold by more than 1e-5 relative, members definite) and B its borderline ones, the GPU
set G must satisfy D <= G <= D u B. Per-object floats of objects in both sets must agree within
1e-4 relative, measured against max(|a|, |b|, floor) with floors 1e-6 /cm for curvatures, 1e-3 for
chi2, 1e-4 rad for angles, 1e-3 GeV for pT, 1e-3 cm for lengths. Track candidates must match
exactly (type, hits, order) except rows that touch a borderline object's hits or lie within
dR < 0.05 of one.
"""
from __future__ import annotations

import math

import numpy as np

REL = 1e-4
FLOOR = {"kappa": 1e-6, "chi2": 1e-3, "angle": 1e-4, "pt": 1e-3, "length": 1e-3, "eta": 1e-4}


def _close(a, b, floor, angle=False, rel=None):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    if angle:
        d = np.abs(np.remainder(a - b + math.pi, 2 * math.pi) - math.pi)
    else:
        d = np.abs(a - b)
    both_inf = np.isinf(a) & np.isinf(b) & (np.sign(a) == np.sign(b))
    scale = np.maximum(np.maximum(np.abs(np.where(np.isinf(a), 0, a)), np.abs(np.where(np.isinf(b), 0, b))), floor)
    return both_inf | (d <= (REL if rel is None else rel) * scale)


def _kappa(R):
    R = np.asarray(R, dtype=np.float64)
    with np.errstate(divide="ignore"):
        return np.where(np.isinf(R), 0.0, 1.0 / R)


def oracle_keys(ref):
    md = ref["md"]
    mdk = [(int(a), int(b)) for a, b in zip(md["hit_lo"], md["hit_up"])]
    ls = ref["ls"]
    lsk = [mdk[a] + mdk[b] for a, b in zip(ls["md_in"], ls["md_out"])]
    t3 = ref["t3"]
    t3k = [mdk[a] + mdk[b] + mdk[c] for a, b, c in zip(t3["md0"], t3["md1"], t3["md2"])]
    t5 = ref["t5"]
    t5k = [sum((mdk[t5[f"md{k}"][i]] for k in range(5)), ()) for i in range(len(t5["md0"]))]
    pt3k = [(int(p),) + t3k[o] for p, o in zip(ref["pt3"]["pls"], ref["pt3"]["obj"])]
    pt5k = [(int(p),) + t5k[o] for p, o in zip(ref["pt5"]["pls"], ref["pt5"]["obj"])]
    return {"md": mdk, "ls": lsk, "t3": t3k, "t5": t5k, "pt3": pt3k, "pt5": pt5k}


def gpu_keys(got):
    mdk = [(int(a), int(b)) for a, b in zip(got["md_hit_lo"], got["md_hit_up"])]
    lsk = [mdk[a] + mdk[b] for a, b in zip(got["ls_md_in"], got["ls_md_out"])]
    ls_in, ls_out = got["ls_md_in"], got["ls_md_out"]
    t3md = [(ls_in[a], ls_out[a], ls_out[b]) for a, b in zip(got["t3_ls_in"], got["t3_ls_out"])]
    t3k = [mdk[a] + mdk[b] + mdk[c] for a, b, c in t3md]
    t5k = [t3k[a] + t3k[b][2:] for a, b in zip(got["t5_t3_in"], got["t5_t3_out"])]
    pt3k = [(int(p),) + t3k[o] for p, o in zip(got["pt3_pls"], got["pt3_t3"])]
    pt5k = [(int(p),) + t5k[o] for p, o in zip(got["pt5_pls"], got["pt5_t5"])]
    return {"md": mdk, "ls": lsk, "t3": t3k, "t5": t5k, "pt3": pt3k, "pt5": pt5k}


# (oracle table, oracle column, gpu field, kind)
FLOAT_CHECKS = {
    "md": [("dphichange", "md_dphichange", "angle"), ("pt_est", "md_pt_est", "pt")],
    "ls": [("z0", "ls_z0", "length"), ("dphi", "ls_dphi", "angle")],
    "t3": [("R", "t3_r", "kappa"), ("xc", "t3_xc", "length"), ("yc", "t3_yc", "length"),
           ("chi2_rz", "t3_chi2_rz", "chi2"), ("pt_est", "t3_pt_est", "pt")],
    "t5": [("kappa_in", "t5_kappa_in", "kappa"), ("kappa_out", "t5_kappa_out", "kappa"),
           ("kappa_fit", "t5_kappa_fit", "kappa"), ("chi2_c", "t5_chi2_c", "chi2"),
           ("chi2_rz", "t5_chi2_rz", "chi2"), ("eta", "t5_eta", "eta"), ("phi", "t5_phi", "angle"),
           ("pt", "t5_pt", "pt")],
    "pt3": [("chi2_xy", "pt3_chi2_xy", "chi2"), ("chi2_rz", "pt3_chi2_rz", "chi2")],
    "pt5": [("chi2_xy", "pt5_chi2_xy", "chi2"), ("chi2_rz", "pt5_chi2_rz", "chi2")],
}


def compare_event(ref, got, ev=None, check_floats=True, rel=None, floor_scale=1.0,
                  rel_stages=("t3", "t5", "pt3", "pt5", "tc_ext")) -> dict:
    """rel / floor_scale: a tighter float tolerance than the shipped 1e-4 (relative) and floors, for
    the stages in rel_stages (those evaluated in double-float)."""
    rep = {"ok": True, "errors": []}
    rk, gk = oracle_keys(ref), gpu_keys(got)
    n_all = 0
    n_border = 0
    tainted_hits = set()
    tainted_etaphi = []
    for stage in ("md", "ls", "t3", "t5", "pt3", "pt5"):
        tab = ref[stage]
        keys = rk[stage]
        D = {k for k, p, d in zip(keys, tab["pass"], tab["definite"]) if p and d}
        B = {k for k, d in zip(keys, tab["definite"]) if not d}
        G = gk[stage]
        Gs = set(G)
        n_all += len(D)
        n_border += len(B)
        for k in B:
            tainted_hits.update(h for h in (k[1:] if stage.startswith("pt") else k))
        if len(Gs) != len(G):
            rep["errors"].append(f"{stage}: duplicate GPU objects")
        missing = D - Gs
        extra = Gs - D - B
        rep[f"n_{stage}"] = len(G)
        rep[f"n_{stage}_oracle"] = len(D)
        if missing or extra:
            rep["errors"].append(f"{stage}: {len(missing)} missing, {len(extra)} extra "
                                 f"(e.g. missing {sorted(missing)[:2]}, extra {sorted(extra)[:2]})")
        if check_floats and FLOAT_CHECKS.get(stage):
            idx = {k: i for i, k in enumerate(keys)}
            pairs = [(idx[k], j) for j, k in enumerate(G) if k in D]
            if pairs:
                oi = np.array([a for a, _ in pairs])
                gi = np.array([b for _, b in pairs])
                for ocol, gcol, kind in FLOAT_CHECKS[stage]:
                    a = np.asarray(tab[ocol])[oi]
                    b = np.asarray(got[gcol], dtype=np.float64)[gi]
                    if kind == "kappa":
                        if ocol == "R":
                            a, b = _kappa(a), _kappa(b)
                    tight = stage in rel_stages
                    ok = _close(a, b, FLOOR[kind] * (floor_scale if tight else 1.0), angle=(kind == "angle"),
                                rel=rel if tight else None)
                    if not ok.all():
                        bad = np.nonzero(~ok)[0][:3]
                        rep["errors"].append(f"{stage}.{ocol}: {int((~ok).sum())} floats differ, e.g. "
                                             f"{[(float(a[i]), float(b[i])) for i in bad]}")
    # borderline T5 / pixel objects taint their eta-phi neighbourhood in the track candidates
    t5 = ref["t5"]
    for i in np.nonzero(~t5["definite"])[0]:
        tainted_etaphi.append((float(t5["eta"][i]), float(t5["phi"][i])))
    if ev is not None:
        for stage in ("pt3", "pt5"):
            for i in np.nonzero(~ref[stage]["definite"])[0]:
                p = int(ref[stage]["pls"][i])
                tainted_etaphi.append((float(ev.pls["eta"][p]), float(ev.pls["phi"][p])))
                tainted_hits.update(int(h) for h in ev.pls["pix_hit"][p])
    rep["n_borderline"] = n_border
    rep["n_objects"] = n_all + n_border
    rep["borderline_fraction"] = n_border / max(1, n_all + n_border)
    # borderline objects must stay below 1e-4 of all objects at every size: below 1e4 objects that
    # allows at most one (the limit rounded up)
    if n_all + n_border > 1e4:
        if rep["borderline_fraction"] >= 1e-4:
            rep["errors"].append(f"borderline fraction {rep['borderline_fraction']:.2e} >= 1e-4")
    elif n_border > 1:
        rep["errors"].append(f"{n_border} borderline objects among {n_all + n_border} (at most 1 below 1e4)")

    # referential integrity of the GPU arrays
    nmd, nls, nt3, nt5 = (len(gk[s]) for s in ("md", "ls", "t3", "t5"))
    for name, arr, n in (("ls_md_in", got["ls_md_in"], nmd), ("ls_md_out", got["ls_md_out"], nmd),
                         ("t3_ls_in", got["t3_ls_in"], nls), ("t3_ls_out", got["t3_ls_out"], nls),
                         ("t5_t3_in", got["t5_t3_in"], nt3), ("t5_t3_out", got["t5_t3_out"], nt3),
                         ("pt3_t3", got["pt3_t3"], nt3), ("pt5_t5", got["pt5_t5"], nt5)):
        a = np.asarray(arr)
        if a.size and (a.min() < 0 or a.max() >= n):
            rep["errors"].append(f"{name} out of range")

    # track candidates
    rtc = ref["tc"]
    r_rows = [(int(rtc["type"][i]),) + tuple(int(rtc[f"hit{k}"][i]) for k in range(14))
              for i in range(len(rtc["type"]))]
    g_rows = [(int(t),) + tuple(int(h) for h in row) for t, row in zip(got["tc_type"], got["tc_hits"])]
    rep["n_tc"] = len(g_rows)
    rep["n_tc_oracle"] = len(r_rows)

    def tainted(row, eta, phi):
        if any(h in tainted_hits for h in row[1:] if h >= 0):
            return True
        for e2, p2 in tainted_etaphi:
            dp = abs(math.remainder(phi - p2, 2 * math.pi))
            if (eta - e2) ** 2 + dp ** 2 < 0.05 ** 2:
                return True
        return False
    if not tainted_hits and not tainted_etaphi:
        if r_rows != g_rows:
            nd = sum(1 for a, b in zip(r_rows, g_rows) if a != b)
            rep["errors"].append(f"tc: lists differ ({len(r_rows)} vs {len(g_rows)} rows, {nd} rows differ)")
    else:
        rc = [r for i, r in enumerate(r_rows) if not tainted(r, rtc["eta"][i], rtc["phi"][i])]
        gc = [r for i, r in enumerate(g_rows) if not tainted(r, got["tc_eta"][i], got["tc_phi"][i])]
        rep["n_tc_tainted"] = len(r_rows) - len(rc)
        if rc != gc:
            rep["errors"].append(f"tc: untainted lists differ ({len(rc)} vs {len(gc)})")
    if r_rows == g_rows and check_floats and r_rows:
        for ocol, gcol, kind in (("pt", "tc_pt", "pt"), ("eta", "tc_eta", "eta"), ("phi", "tc_phi", "angle")):
            ok = _close(rtc[ocol], got[gcol], FLOOR[kind], angle=(kind == "angle"))
            if not ok.all():
                rep["errors"].append(f"tc.{ocol}: {int((~ok).sum())} floats differ")

    # track extensions (Sec. 2.5.1), row by row on the rows that match: the MDs added, their hits
    # and the extending T3 (by its hit key) exactly, the fit chi2 within the float tolerance; rows
    # where one of the oracle's candidate T3 was borderline are skipped
    ext = ref.get("tc_ext")
    if ext is not None and "tc_ext_n_md" in got:
        ridx = [i for i in range(len(r_rows)) if not tainted(r_rows[i], rtc["eta"][i], rtc["phi"][i])]
        gidx = [i for i in range(len(g_rows)) if not tainted(g_rows[i], got["tc_eta"][i], got["tc_phi"][i])]
        n_cmp = n_ext = n_bad = 0
        if [r_rows[i] for i in ridx] == [g_rows[i] for i in gidx]:
            for i, j in zip(ridx, gidx):
                if not ext["definite"][i]:
                    continue
                n_cmp += 1
                ro = (int(ext["n_add"][i]),) + tuple(int(ext[f"hit{k}"][i]) for k in range(4))
                go = (int(got["tc_ext_n_md"][j]),) + tuple(int(h) for h in got["tc_ext_hits"][j])
                same = ro == go
                if same and ro[0] > 0:
                    n_ext += 1
                    gt = int(got["tc_ext_t3"][j])
                    same = 0 <= gt < len(gk["t3"]) and gk["t3"][gt] == rk["t3"][int(ext["t3"][i])]
                    if same and check_floats:
                        tight = "tc_ext" in rel_stages
                        fl = FLOOR["chi2"] * (floor_scale if tight else 1.0)
                        r_ = rel if tight else None
                        same = bool(_close(ext["chi2_c"][i], got["tc_ext_chi2_c"][j], fl, rel=r_)) and \
                            bool(_close(ext["chi2_rz"][i], got["tc_ext_chi2_rz"][j], fl, rel=r_))
                n_bad += not same
        rep["n_tc_ext"] = n_ext
        rep["n_tc_ext_compared"] = n_cmp
        if n_bad:
            rep["errors"].append(f"tc_ext: {n_bad} of {n_cmp} rows differ")
    rep["ok"] = not rep["errors"]
    return rep


def binning_matches(ref, got_order, got_offsets) -> bool:
    return np.array_equal(ref["order"], got_order) and np.array_equal(ref["offsets"], got_offsets)
