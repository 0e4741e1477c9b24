"""Pins of the CPU oracle against what the paper and the mathematics fix.

* closed forms: circumcircle (Triplet circle, Sec. 2.3), Karimaki's circle fit (Quintuplet global
  fit, Sec. 2.3) against the exact circle and a geometric least-squares fit, the weighted r-z line
  fit against numpy.polyfit, the pixel-seed bin;
* single-helix invariants: one Mini-Doublet per crossed module (Sec. 2.2), LS/T3/T5 chain along the
  crossed modules, object sizes 2/4/6/10 hits (Sec. 2.1), MD pT estimate, the pT threshold turn-on;
* referential integrity of member indices;
* the Track-Candidate rules (Sec. 2.5) re-derived independently in Python on the oracle's objects.
"""
import math

import numpy as np
import pytest
from scipy.optimize import least_squares

import oracle
from paper_2207_08207_gb300 import gen


# ------------------------------------------------------------------------------------------------
# closed forms
# ------------------------------------------------------------------------------------------------
def test_circumcircle_closed_form():
    rng = np.random.default_rng(1)
    for _ in range(200):
        p = rng.uniform(-100, 100, 6)
        xc, yc, R = oracle.circumcircle(p)
        a, b, c = p[0:2], p[2:4], p[4:6]
        # centre solves |u-a|^2 = |u-b|^2 = |u-c|^2 (two linear equations)
        A = np.array([2 * (b - a), 2 * (c - a)])
        rhs = np.array([b @ b - a @ a, c @ c - a @ a])
        u = np.linalg.solve(A, rhs)
        assert np.allclose([xc, yc], u, rtol=1e-9, atol=1e-9)
        for q in (a, b, c):
            assert abs(np.hypot(*(q - u)) - R) < 1e-8 * max(1.0, R)
    xc, yc, R = oracle.circumcircle(np.array([0.0, 0.0, 1.0, 1.0, 2.0, 2.0]))
    assert math.isinf(R)


def _circle_points(q, R, phi0, n=5, d0=0.0, spread=(23.0, 110.0)):
    h = gen.Helices(np.array([q]), np.array([R]), np.array([phi0]), np.array([0.0]),
                    np.array([d0]), np.array([0.0]))
    rs = np.linspace(*spread, n)
    pts = []
    for r in rs:
        p1, p2 = gen.cylinder_psi(h, r)
        x, y, _ = h.position(np.array([min(p1[0], p2[0])]))
        pts.append((x[0], y[0]))
    return np.array(pts)


@pytest.mark.parametrize("q", [-1.0, 1.0])
@pytest.mark.parametrize("R", [70.0, 300.0, 3000.0, 1e5])
def test_karimaki_exact_circle(q, R):
    pts = _circle_points(q, R, 0.7, d0=0.05)
    rho, phi, d, chi2 = oracle.karimaki(pts[:, 0], pts[:, 1])
    # the helix convention: centre to the right of the direction for q > 0, so rho = q / R
    assert abs(rho - q / R) <= 1e-6 * abs(q / R) + 1e-12
    assert abs(math.remainder(phi - 0.7, 2 * math.pi)) < 1e-6
    assert chi2 < 1e-16
    assert abs(abs(d) - 0.05) < 1e-6


def test_karimaki_vs_geometric_fit():
    rng = np.random.default_rng(3)
    for _ in range(50):
        q = rng.choice([-1.0, 1.0])
        R = rng.uniform(70, 2000)
        pts = _circle_points(q, R, rng.uniform(-3, 3))
        pts += rng.normal(0, 0.003, pts.shape)
        rho, phi, d, chi2 = oracle.karimaki(pts[:, 0], pts[:, 1])
        xc0, yc0 = (1 / rho + d) * math.sin(phi), -(1 / rho + d) * math.cos(phi)

        def res(v):
            return np.hypot(pts[:, 0] - v[0], pts[:, 1] - v[1]) - v[2]
        fit = least_squares(res, [xc0, yc0, 1 / abs(rho)], xtol=1e-15, ftol=1e-15, gtol=1e-15)
        chi2_geo = float(np.sum(fit.fun ** 2))
        assert chi2 >= chi2_geo * (1 - 1e-9) - 1e-18
        assert chi2 <= chi2_geo * 1.05 + 1e-12
        assert abs(1 / fit.x[2] - abs(rho)) <= 0.01 * abs(rho)


def test_line_fit_matches_polyfit():
    rng = np.random.default_rng(4)
    for n in (3, 5):
        s = np.sort(rng.uniform(20, 120, n))
        z = 3.0 + 1.7 * s + rng.normal(0, 0.1, n)
        sig = rng.uniform(0.05, 0.3, n)
        chi2, slope = oracle.line_fit(s, z, sig)
        b, a = np.polyfit(s, z, 1, w=1 / sig)
        assert abs(slope - b) < 1e-9
        assert abs(chi2 - np.sum(((z - a - b * s) / sig) ** 2)) < 1e-9


def test_pixel_bin_closed_form():
    assert oracle.pixel_bin(0.0, 0.0, 1) == (50 * 128 + 0) * 2 + 1
    assert oracle.pixel_bin(-2.5, 0.0, -1) == 0
    assert oracle.pixel_bin(2.5, 0.0, 1) == -1
    assert oracle.pixel_bin(0.049, 3.0, -1) == (50 * 128 + int(3.0 * 64 / math.pi)) * 2
    assert oracle.pixel_bin(0.051, -0.1, 1) == (51 * 128 + int((2 * math.pi - 0.1) * 64 / math.pi)) * 2 + 1
    rng = np.random.default_rng(5)
    for _ in range(500):
        e = np.float32(rng.uniform(-2.6, 2.6))
        p = np.float32(rng.uniform(-math.pi, math.pi))
        c = int(rng.choice([-1, 1]))
        assert oracle.pixel_bin(e, p, c) == int(gen.pixel_bin_of(e, p, c))


def test_constants_table():
    c = oracle.constants()
    f = np.float32
    assert c[0] == float(f(0.0114)) and c[1] == float(f(0.8)) and c[20] == float(f(0.01))
    assert c[-1] == 7


# ------------------------------------------------------------------------------------------------
# single helices
# ------------------------------------------------------------------------------------------------
def _crossed_modules(det, ev_sensor):
    s = np.asarray(ev_sensor)
    mods = s // 2
    both = [m for m in np.unique(mods) if (2 * m in s) and (2 * m + 1 in s)]
    return sorted(both)


def _keys(res, table):
    md = res["md"]
    def mdh(i):
        return (int(md["hit_lo"][i]), int(md["hit_up"][i]))
    if table == "md":
        return {mdh(i) for i in range(len(md["module"]))}
    if table == "ls":
        ls = res["ls"]
        return {mdh(a) + mdh(b) for a, b in zip(ls["md_in"], ls["md_out"])}
    if table == "t3":
        t = res["t3"]
        return {mdh(a) + mdh(b) + mdh(c) for a, b, c in zip(t["md0"], t["md1"], t["md2"])}
    if table == "t5":
        t = res["t5"]
        return {sum((mdh(t[f"md{k}"][i]) for k in range(5)), ()) for i in range(len(t["md0"]))}


@pytest.mark.parametrize("pt", [1.0, 2.0, 5.0, 10.0])
@pytest.mark.parametrize("q", [-1, 1])
@pytest.mark.parametrize("eta", [0.0, 0.5, 0.9])
def test_single_helix_chain(pt, q, eta):
    det = gen.make_detector(barrel_only=True, pt_thr=0.8)
    ev = gen.single_helix_event(det.geom, q, pt, eta, phi0=0.4, z0=1.0)
    res = oracle.run(det, ev)
    md = res["md"]
    crossed = _crossed_modules(det, ev.sensor)
    # exactly one MD per module whose two sensors were both crossed, and none elsewhere
    assert sorted(md["module"].tolist()) == crossed
    assert md["pass"].all() and md["definite"].all()
    # MD pT estimate on noise-free barrel hits: the hit-pair direction is the chord from r_l to
    # r_l + spacing, so to first order pt_est = pT * r_l / (r_l + spacing)
    rl = md["r"]
    sp = det.geom.spacing[md["module"]]
    assert np.all(np.abs(md["pt_est"] / (pt * rl / (rl + sp)) - 1.0) < 2e-3)
    assert np.all(np.abs(md["pt_est"] / pt - 1.0) < 0.012)
    # LS link consecutive crossed modules; T3/T5 chain along them
    layer = det.geom.layer[md["module"]]
    order = np.argsort(layer)
    ls = res["ls"]
    expected_ls = {(order[k], order[k + 1]) for k in range(len(order) - 1)
                   if layer[order[k + 1]] == layer[order[k]] + 1}
    assert {(int(a), int(b)) for a, b in zip(ls["md_in"], ls["md_out"])} == expected_ls
    n_ls = len(expected_ls)
    assert len(res["t3"]["md0"]) == max(0, n_ls - 1) if n_ls == len(order) - 1 else True
    t3 = res["t3"]
    for i in range(len(t3["md0"])):
        assert layer[t3["md1"][i]] == layer[t3["md0"][i]] + 1
        assert layer[t3["md2"][i]] == layer[t3["md1"][i]] + 1
    t5 = res["t5"]
    for i in range(len(t5["md0"])):
        ls_ = [layer[t5[f"md{k}"][i]] for k in range(5)]
        assert ls_ == list(range(ls_[0], ls_[0] + 5))
    # 6 crossed barrel layers give 5 LS, 4 T3, 2 T5 and one T5 track candidate
    if len(crossed) == 6:
        assert len(ls["md_in"]) == 5 and len(t3["md0"]) == 4 and len(t5["md0"]) == 2
        tc = res["tc"]
        assert len(tc["type"]) == 1 and tc["type"][0] == 2
        assert abs(tc["pt"][0] / pt - 1) < 1e-3


def test_below_threshold_no_outer_md():
    det = gen.make_detector(barrel_only=True, pt_thr=0.8)
    for q in (-1, 1):
        ev = gen.single_helix_event(det.geom, q, 0.5, 0.2, phi0=1.0)
        res = oracle.run(det, ev)
        layers = det.geom.layer[res["md"]["module"]]
        assert not np.any(layers >= 4)
        # the helix does cross the outer layers
        assert np.any(det.geom.layer[ev.sensor // 2] >= 4)


def test_at_threshold_passes():
    det = gen.make_detector(barrel_only=True, pt_thr=0.8)
    ev = gen.single_helix_event(det.geom, 1, 0.8 * 1.0001, 0.1, phi0=2.0)
    res = oracle.run(det, ev)
    assert sorted(res["md"]["module"].tolist()) == _crossed_modules(det, ev.sensor)


def test_displaced_vertex_fails_pointing():
    det = gen.make_detector(barrel_only=True, pt_thr=0.8)
    ok = oracle.run(det, gen.single_helix_event(det.geom, 1, 3.0, 0.3, z0=0.0))
    bad = oracle.run(det, gen.single_helix_event(det.geom, 1, 3.0, 0.3, z0=45.0))
    assert len(ok["ls"]["md_in"]) >= 4
    assert len(bad["md"]["module"]) >= 4     # MDs still form (local cut)
    assert len(bad["ls"]["md_in"]) == 0      # LS r-z pointing rejects z0 far outside the luminous region


def test_smeared_helix_high_efficiency():
    det = gen.make_detector(barrel_only=True, pt_thr=0.8)
    found = 0
    for seed in range(20):
        ev = gen.single_helix_event(det.geom, 1 if seed % 2 else -1, 1.5 + seed, 0.3, phi0=0.1 * seed,
                                    smear=True, seed=seed)
        res = oracle.run(det, ev)
        found += len(res["tc"]["type"]) == 1
    assert found >= 18


# ------------------------------------------------------------------------------------------------
# integrity and Track-Candidate rules on a small PU event
# ------------------------------------------------------------------------------------------------
@pytest.fixture(scope="module")
def small_pu():
    det, ev = gen.small_event(400, seed=77)
    return det, ev, oracle.run(det, ev)


def test_referential_integrity(small_pu):
    det, ev, r = small_pu
    md, ls, t3, t5 = r["md"], r["ls"], r["t3"], r["t5"]
    nmd, nls, nt3 = len(md["module"]), len(ls["md_in"]), len(t3["md0"])
    assert np.all((md["hit_lo"] >= 0) & (md["hit_lo"] < ev.n_hits))
    assert np.all(ev.sensor[md["hit_lo"]] == 2 * md["module"])
    assert np.all(ev.sensor[md["hit_up"]] == 2 * md["module"] + 1)
    assert np.all((ls["md_in"] < nmd) & (ls["md_out"] < nmd))
    co, ct = det.conn_off, det.conn_tgt
    for a, b in zip(ls["md_in"], ls["md_out"]):
        assert md["module"][b] in ct[co[md["module"][a]]:co[md["module"][a] + 1]]
    assert np.all((t3["ls_in"] < nls) & (t3["ls_out"] < nls))
    assert np.all(ls["md_out"][t3["ls_in"]] == ls["md_in"][t3["ls_out"]])
    assert np.all(t3["md0"] == ls["md_in"][t3["ls_in"]])
    assert np.all(t3["md2"] == ls["md_out"][t3["ls_out"]])
    assert np.all((t5["t3_in"] < nt3) & (t5["t3_out"] < nt3))
    assert np.all(t3["md2"][t5["t3_in"]] == t3["md0"][t5["t3_out"]])
    for name, obj in (("pt3", nt3), ("pt5", len(t5["md0"]))):
        assert np.all(r[name]["obj"] < obj) and np.all(r[name]["pls"] < ev.n_pls)


def test_track_candidate_rules(small_pu):
    """Sec. 2.5 re-derived in Python: one best pT5/pT3 per seed, non-greedy T5 duplicate removal,
    the pT5 -> pT3 -> T5 -> pLS order with eta-phi cross-cleaning, and the hit counts per type."""
    det, ev, r = small_pu
    md, t3, t5, tc = r["md"], r["t3"], r["t5"], r["tc"]
    pls = ev.pls

    def mdhits(ids):
        return [h for i in ids for h in (int(md["hit_lo"][i]), int(md["hit_up"][i]))]
    t5h = [mdhits([t5[f"md{k}"][i] for k in range(5)]) for i in range(len(t5["md0"]))]
    t3h = [mdhits([t3[f"md{k}"][i] for k in range(3)]) for i in range(len(t3["md0"]))]

    def best(table, hits_of):
        b = {}
        for i in range(len(table["pls"])):
            if not table["pass"][i]:
                continue
            p = int(table["pls"][i])
            key = (np.float32(table["score"][i]), tuple(sorted(list(pls["pix_hit"][p]) + hits_of[table["obj"][i]])))
            if p not in b or key < b[p][0]:
                b[p] = (key, i)
        return b
    b5, b3 = best(r["pt5"], t5h), best(r["pt3"], t3h)

    kept = []
    for a in range(len(t5h)):
        if not t5["pass"][a]:
            continue
        ka = (np.float32(t5["chi2_c"][a]), tuple(sorted(t5h[a])))
        drop = any(t5["pass"][b] and b != a and len(set(t5h[a]) & set(t5h[b])) >= 7 and
                   (np.float32(t5["chi2_c"][b]), tuple(sorted(t5h[b]))) < ka for b in range(len(t5h)))
        if not drop:
            kept.append(a)
    assert kept == list(np.nonzero(r["t5_kept"])[0])

    def close(e1, p1, e2, p2):
        de = float(e1) - float(e2)
        dp = float(p1) - float(p2)
        if dp > math.pi:
            dp -= 2 * math.pi
        if dp <= -math.pi:
            dp += 2 * math.pi
        return de * de + dp * dp < float(np.float32(0.01)) ** 2

    acc = []
    exp5 = [(0, tuple(sorted(list(pls["pix_hit"][p]) + t5h[r["pt5"]["obj"][i]])), pls["eta"][p], pls["phi"][p])
            for p, (_, i) in b5.items()]
    acc += exp5
    exp3 = []
    for p, (_, i) in b3.items():
        if p in b5 or any(close(pls["eta"][p], pls["phi"][p], e, f) for *_, e, f in exp5):
            continue
        exp3.append((1, tuple(sorted(list(pls["pix_hit"][p]) + t3h[r["pt3"]["obj"][i]])), pls["eta"][p], pls["phi"][p]))
    acc += exp3
    expt5 = []
    for a in kept:
        e, f = np.float32(t5["eta"][a]), np.float32(t5["phi"][a])
        if any(close(e, f, e2, f2) for *_, e2, f2 in acc):
            continue
        expt5.append((2, tuple(sorted(t5h[a])), e, f))
    acc += expt5
    member = set(r["pt3"]["pls"][r["pt3"]["pass"]]) | set(r["pt5"]["pls"][r["pt5"]["pass"]])
    expl = []
    for p in range(ev.n_pls):
        if p in member or any(close(pls["eta"][p], pls["phi"][p], e, f) for *_, e, f in acc):
            continue
        expl.append((3, tuple(sorted(pls["pix_hit"][p])), 0, 0))
    expected = [(t, k) for lst in (exp5, exp3, expt5, expl) for t, k, *_ in sorted(lst, key=lambda c: c[1])]
    got = []
    for i in range(len(tc["type"])):
        hits = [int(tc[f"hit{k}"][i]) for k in range(14) if tc[f"hit{k}"][i] >= 0]
        got.append((int(tc["type"][i]), tuple(sorted(hits))))
        assert len(hits) == {0: 14, 1: 10, 2: 10, 3: 4}[int(tc["type"][i])]
    assert got == expected
    assert len(exp5) > 0 and len(exp3) > 0 and len(expl) > 0
