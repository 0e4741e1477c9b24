"""Pins of the oracle's endcap branches, its pixel-seed (pT3 / pT5) chi2 terms and the edge of the
Line-Segment pointing window, against geometry and statistics fixed outside the oracle.

* Endcap single helices (Sec. 2.2, 2.3): a noise-free helix through the disks gives one Mini-Doublet
  per crossed module; the endcap MD's dPhiChange is minus the charge times half the turning angle
  to the lower hit, so sin|dPhiChange| = r / 2R and the MD pT estimate is the true pT, within the
  float32 rounding of the hit coordinates carried through |z| / spacing; every module-map-connected
  pair of crossed modules forms an LS, every LS pair sharing an MD a T3 and every T3 pair sharing
  an MD a T5, with r-z chi2 ~ 0 under the sigma_r |slope| endcap model, the fitted curvature q / R,
  eta the helix's and phi its direction at closest approach.
* Pixel seeds (Sec. 2.4): a seed holding a helix's true parameters gives chi2 ~ 0 for the T3 and
  T5 of that helix; the opposite-charge seed's circle is the true circle mirrored across the seed
  direction, and its per-anchor distances equal those of that mirrored circle; over seeds smeared
  as the generator smears them (1 % pT, 1 mrad in phi and theta) and hits smeared by the stated
  resolutions, each anchor's squared residual over its variance averages 1, which fixes the
  variance model (hit resolution plus the seed's direction and curvature uncertainty carried to
  the anchor radius) term by term.
* LS pointing window edge (Sec. 2.2): tracks from z0 just inside and just outside
  +-(z_lum + n_sigma sigma_z0), with sigma_z0 obtained here by numerical error propagation of the
  straight-line intercept from the hit resolutions, are accepted or rejected as the reading
  predicts for a straight track (z0 of the anchors' line = z0) and for a helix at the threshold
  radius (z0 in arc length = z0).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2207_08207_gb300 import gen

F32_EPS = 2.0 ** -24
N_SIGMA, Z_LUM, SIGMA_Z, SIGMA_R = 3.0, 15.0, 0.1, 0.1


@pytest.fixture(scope="module")
def det():
    return gen.make_detector(barrel_only=False, pt_thr=0.8)


def _crossings(det, q, pt, eta, phi0, z0, d0=0.0):
    """Lower-sensor crossings of one helix in turning order: (module, x, y, z) rows, plus the
    modules whose two sensors were both crossed."""
    h = gen.Helices(np.array([float(q)]), np.array([pt / gen.K_B]), np.array([phi0]),
                    np.array([math.sinh(eta)]), np.array([d0]), np.array([z0]))
    _, si, psi, mod, x, y, z = gen.crossings(det.geom, h)
    surfs = gen.surfaces(False)
    sens = np.array([surfs[i].sensor for i in si])
    both = {int(m) for m in mod[sens == 0]} & {int(m) for m in mod[sens == 1]}
    low = sens == 0
    order = np.argsort(psi[low])
    rows = [(int(m), float(a), float(b), float(c)) for m, a, b, c in
            zip(mod[low][order], x[low][order], y[low][order], z[low][order]) if int(m) in both]
    return h, rows


def _expected_chain(det, mods):
    """Objects a noise-free helix above threshold must build: LS = every ordered pair of its crossed
    modules (in crossing order) that the module map connects; T3 / T5 = every pair sharing an MD."""
    co, ct = det.conn_off, det.conn_tgt
    ls = {(i, j) for i in range(len(mods)) for j in range(i + 1, len(mods))
          if mods[j] in ct[co[mods[i]]:co[mods[i] + 1]]}
    t3 = {(a, b, c) for (a, b) in ls for (b2, c) in ls if b2 == b}
    t5 = {t[:3] + u[1:] for t in t3 for u in t3 if u[0] == t[2]}
    return ls, t3, t5


@pytest.mark.parametrize("pt", [1.0, 2.0, 5.0, 10.0])
@pytest.mark.parametrize("q", [-1, 1])
@pytest.mark.parametrize("eta", [1.5, 1.9, 2.3, -1.9])
def test_endcap_single_helix_chain(det, pt, q, eta):
    phi0 = 0.4
    ev = gen.single_helix_event(det.geom, q, pt, eta, phi0=phi0, z0=0.0)
    hel, rows = _crossings(det, q, pt, eta, phi0, 0.0)
    res = oracle.run(det, ev)
    md = res["md"]
    g = det.geom
    # one definite MD per module whose two sensors were crossed, in the same modules
    assert sorted(md["module"].tolist()) == sorted(m for m, *_ in rows)
    assert md["pass"].all() and md["definite"].all()
    R = pt / gen.K_B
    ec = g.subdet[md["module"]] == gen.SUBDET_ENDCAP
    assert ec.sum() >= 3
    for i in np.nonzero(ec)[0]:
        r, az = float(md["r"][i]), abs(float(md["z"][i]))
        delta = float(g.spacing[md["module"][i]])
        dpc = float(md["dphichange"][i])
        # float32 hit coordinates move each azimuth by <= 2^-24 rad; dPhiChange scales it by |z|/delta
        tol = 2.5 * F32_EPS * az / delta + 1e-9
        assert np.sign(dpc) == -q
        assert abs(abs(math.sin(dpc)) - r / (2 * R)) <= tol
        assert abs(md["pt_est"][i] - pt) <= pt * tol / abs(math.tan(dpc)) + 1e-6
    # the module map's connections among the crossed modules define the whole chain
    mods = [m for m, *_ in rows]
    pos = {m: k for k, m in enumerate(mods)}
    mdpos = np.array([pos[int(m)] for m in md["module"]])
    ls_e, t3_e, t5_e = _expected_chain(det, mods)
    ls = res["ls"]
    assert {(int(mdpos[a]), int(mdpos[b])) for a, b in zip(ls["md_in"], ls["md_out"])} == ls_e
    t3 = res["t3"]
    assert {tuple(int(mdpos[t3[f"md{k}"][i]]) for k in range(3)) for i in range(len(t3["md0"]))} == t3_e
    t5 = res["t5"]
    assert {tuple(int(mdpos[t5[f"md{k}"][i]]) for k in range(5)) for i in range(len(t5["md0"]))} == t5_e
    assert len(t5_e) >= 1
    assert ls["pass"].all() and t3["pass"].all() and t5["pass"].all()
    assert np.all(t3["chi2_rz"] <= 1e-6) and np.all(t5["chi2_rz"] <= 1e-6)
    assert np.all(t5["chi2_c"] <= 1e-5)
    # T5 parameters against the helix: curvature q / R with an error bounded by the float32
    # coordinate rounding over the sagitta of the five anchors, eta, and phi at closest approach
    for i in range(len(t5["md0"])):
        idx = [int(t5[f"md{k}"][i]) for k in range(5)]
        px, py = md["x"][idx], md["y"][idx]
        chord = math.hypot(px[-1] - px[0], py[-1] - py[0])
        sag = chord * chord / (8 * R)
        rtol = 40 * F32_EPS * float(np.max(md["r"][idx])) / sag + 1e-9
        assert abs(t5["kappa_fit"][i] - q / R) <= rtol / R
        assert abs(t5["pt"][i] / pt - 1) <= 2 * rtol
        assert abs(t5["eta"][i] - eta) <= 1e-5
        assert abs(math.remainder(t5["phi"][i] - phi0, 2 * math.pi)) <= 1e-5
    # T3 circles: centre and radius of the helix's circle
    for i in range(len(t3["md0"])):
        assert abs(t3["R"][i] / R - 1) <= 1e-3
        assert math.hypot(t3["xc"][i] - hel.cx[0], t3["yc"][i] - hel.cy[0]) <= 1e-3 * R


# ------------------------------------------------------------------------------------------------
# pixel seeds
# ------------------------------------------------------------------------------------------------
def _seed(q, pt, eta, phi0, z0, x0=0.0, y0=0.0, hit0=10_000):
    s = np.zeros(1, dtype=gen.PLS_DTYPE)
    s["pt"], s["eta"], s["phi"] = pt, eta, phi0
    s["x0"], s["y0"], s["z0"] = x0, y0, z0
    s["charge"] = q
    s["pix_hit"] = hit0 + np.arange(4)
    return s


@pytest.mark.parametrize("eta", [0.3, 1.5, 1.9, -2.3])
@pytest.mark.parametrize("q", [-1, 1])
@pytest.mark.parametrize("pt", [1.0, 3.0, 10.0])
def test_true_seed_chi2_vanishes(det, eta, q, pt):
    phi0, z0 = -2.1, 2.0
    ev = gen.single_helix_event(det.geom, q, pt, eta, phi0=phi0, z0=z0)
    ev.pls = _seed(q, pt, eta, phi0, z0, hit0=ev.n_hits)
    res = oracle.run(det, ev)
    for name in ("pt3", "pt5"):
        tab = res[name]
        assert len(tab["pls"]) >= 1, name
        assert tab["pass"].all() and tab["definite"].all()
        assert np.all(tab["chi2_xy"] <= 1e-6) and np.all(tab["chi2_rz"] <= 1e-6), name
    tc = res["tc"]
    assert list(tc["type"]) == [0]   # one pT5 track candidate, nothing else
    # the opposite charge: no pixel object at all
    ev.pls = _seed(-q, pt, eta, phi0, z0, hit0=ev.n_hits)
    res = oracle.run(det, ev)
    assert len(res["pt3"]["pls"]) == 0 and len(res["pt5"]["pls"]) == 0


@pytest.mark.parametrize("eta", [0.3, 2.0])
@pytest.mark.parametrize("q", [-1, 1])
def test_opposite_charge_seed_is_the_mirrored_circle(det, eta, q):
    pt, phi0, z0, d0 = 1.5, 0.9, -1.0, 0.02
    hel, rows = _crossings(det, q, pt, eta, phi0, z0, d0=d0)
    x = np.array([r[1] for r in rows])
    y = np.array([r[2] for r in rows])
    z = np.array([r[3] for r in rows])
    ec = det.geom.subdet[[r[0] for r in rows]] == gen.SUBDET_ENDCAP
    x0, y0 = float(hel.x0[0]), float(hel.y0[0])
    s_true = _seed(q, pt, eta, phi0, z0, x0, y0)
    t, (cxy, crz) = oracle.seed_terms(s_true, x, y, z, ec)
    # on the circle, to the float32 rounding of the seed record (~1e-6 cm); on the r-z line to
    # O(d0 cot theta), since the arc length is measured from the origin (d0 = 0 pins it at ~0 above)
    assert np.all(np.abs(t[:, 0]) <= 2e-5)
    assert np.all(np.abs(t[:, 2]) <= abs(d0 * math.sinh(eta)) + 1e-5)
    # mirror the true centre across the seed's direction line through (x0, y0)
    u = np.array([math.cos(phi0), math.sin(phi0)])
    p0 = np.array([x0, y0])
    c = np.array([hel.cx[0], hel.cy[0]])
    cm = 2 * (p0 + ((c - p0) @ u) * u) - c
    R = pt / gen.K_B
    dist = np.hypot(x - cm[0], y - cm[1]) - R
    s_opp = _seed(-q, pt, eta, phi0, z0, x0, y0)
    t2, (cxy2, crz2) = oracle.seed_terms(s_opp, x, y, z, ec)
    assert np.allclose(t2[:, 0], dist, rtol=0, atol=2e-5)
    assert np.allclose(t2[:, 1], t[:, 1]) and np.allclose(t2[:, 2], t[:, 2])
    assert abs(cxy2 - float(np.sum(t2[:, 0] ** 2 / t2[:, 1]))) <= 1e-9 * cxy2
    assert cxy2 > 25.0   # far beyond both pixel-object cuts


@pytest.mark.parametrize("region", ["barrel", "endcap"])
def test_seed_variance_model_matches_the_smearing(region):
    """Mean of residual^2 / variance per anchor over seeds and hits smeared as generated."""
    g = gen.make_geometry(False)
    rng = np.random.default_rng(2024 if region == "barrel" else 2025)
    n = 1500
    pt = gen._powerlaw_pt(rng, n, 0.8)
    if region == "barrel":
        eta = rng.uniform(-0.8, 0.8, n)
    else:
        eta = rng.choice([-1.0, 1.0], n) * rng.uniform(1.8, 2.4, n)
    phi0 = rng.uniform(-math.pi, math.pi, n)
    z0 = rng.normal(0, 5, n)
    d0 = rng.normal(0, 0.01, n)
    q = rng.choice([-1, 1], n)
    ev = gen.simulate(g, rng, q, pt, phi0, eta, d0, z0, eff=1.0, pls_min_pt=0.8, shuffle=False)
    lower = ev.sensor % 2 == 0
    xy, rz, lowpt = [], [], []
    for k, p in enumerate(ev.pls_particle):
        sel = np.nonzero(lower & (ev.hit_particle == p))[0]
        if sel.size < 3:
            continue
        sel = sel[np.argsort(np.abs(ev.z[sel]) + np.hypot(ev.x[sel], ev.y[sel]))[:5]]
        ec = g.subdet[ev.sensor[sel] // 2] == gen.SUBDET_ENDCAP
        if region == "barrel" and ec.any():
            continue
        t, _ = oracle.seed_terms(ev.pls[k], ev.x[sel], ev.y[sel], ev.z[sel], ec)
        xy += list(t[:, 0] ** 2 / t[:, 1])
        rz += list(t[:, 2] ** 2 / t[:, 3])
        lowpt += [pt[p] < 1.5] * sel.size
    xy, rz, lowpt = np.array(xy), np.array(rz), np.array(lowpt)
    assert xy.size > 3000
    hi = 1.12 if region == "barrel" else 1.2   # endcap r smearing adds an unmodelled r.sin(alpha) term
    assert 0.9 <= xy.mean() <= hi, xy.mean()
    assert 0.9 <= rz.mean() <= 1.12, rz.mean()
    # the curvature term dominates at low pT: the mean stays ~1 there too
    assert 0.85 <= xy[lowpt].mean() <= hi + 0.05, xy[lowpt].mean()


# ------------------------------------------------------------------------------------------------
# edge of the LS pointing window
# ------------------------------------------------------------------------------------------------
def _sigma_z0(r1, z1, r2, z2, ec1, ec2):
    """Resolution of the intercept at r = 0 of the line through two anchors, by numerical error
    propagation: barrel anchors carry sigma_z in z, endcap anchors sigma_r in r."""
    def z0(v):
        return np.polyfit([v[0], v[2]], [v[1], v[3]], 1)[1]
    v = np.array([r1, z1, r2, z2], dtype=np.float64)
    sig = np.array([SIGMA_R if ec1 else 0.0, 0.0 if ec1 else SIGMA_Z,
                    SIGMA_R if ec2 else 0.0, 0.0 if ec2 else SIGMA_Z])
    var = 0.0
    for k in range(4):
        if sig[k] == 0:
            continue
        h = 1e-4
        dv = np.zeros(4)
        dv[k] = h
        der = (z0(v + dv) - z0(v - dv)) / (2 * h)
        var += (der * sig[k]) ** 2
    return math.sqrt(var)


def _pair_ls(det, res, m1, m2):
    md = res["md"]
    mods = md["module"]
    i1 = np.nonzero(mods == m1)[0]
    i2 = np.nonzero(mods == m2)[0]
    assert i1.size == 1 and i2.size == 1
    ls = res["ls"]
    return any(a == i1[0] and b == i2[0] for a, b in zip(ls["md_in"], ls["md_out"]))


@pytest.mark.parametrize("case", ["barrel", "endcap"])
@pytest.mark.parametrize("kind", ["straight", "threshold"])
@pytest.mark.parametrize("side", [-1, 1])
@pytest.mark.parametrize("cot_sign", [-1, 1])
def test_ls_pointing_window_edge(det, case, kind, side, cot_sign):
    pt = 1e4 if kind == "straight" else 0.8
    eta0 = 0.5 if case == "barrel" else 2.0
    eta = cot_sign * eta0
    eps = 2e-3
    q, phi0 = 1, 0.7
    g = det.geom
    # the first two barrel (or endcap) lower-sensor surfaces the track crosses carry the LS under test
    L = Z_LUM + 1.0
    for _ in range(4):   # sigma_z0 depends on z0 for endcap anchors: iterate to the edge
        z0 = side * (L + eps)
        _, rows = _crossings(det, q, pt, eta, phi0, z0)
        rows = [r for r in rows if (g.subdet[r[0]] == 1) == (case == "endcap")]
        (m1, x1, y1, z1), (m2, x2, y2, z2) = rows[0], rows[1]
        ec1, ec2 = g.subdet[m1] == 1, g.subdet[m2] == 1
        r1, r2 = math.hypot(x1, y1), math.hypot(x2, y2)
        L = Z_LUM + N_SIGMA * _sigma_z0(r1, z1, r2, z2, ec1, ec2)
    co, ct = det.conn_off, det.conn_tgt
    assert m2 in ct[co[m1]:co[m1 + 1]]
    for inside in (True, False):
        z0 = side * (L - eps if inside else L + eps)
        ev = gen.single_helix_event(g, q, pt, eta, phi0=phi0, z0=z0)
        _, rows2 = _crossings(det, q, pt, eta, phi0, z0)
        rows2 = [r for r in rows2 if (g.subdet[r[0]] == 1) == (case == "endcap")]
        assert (rows2[0][0], rows2[1][0]) == (m1, m2)
        res = oracle.run(det, ev)
        got = _pair_ls(det, res, m1, m2)
        if inside:
            expect = True
        else:
            # z0 outside the window on the side of `side`. The anchors' straight-line intercept and
            # the threshold-helix (arc length) intercept differ by cot * X with X > 0 (arc length
            # grows faster than r): for a straight track the line intercept is z0 and the arc one
            # is z0 + cot X; for the threshold helix the arc intercept is z0 and the line one
            # z0 - cot X. The LS exists iff the other intercept moves back inside.
            moves_in = (cot_sign == -side) if kind == "straight" else (cot_sign == side)
            expect = moves_in
        assert got == expect, (case, kind, side, cot_sign, inside, z0, L)


# ------------------------------------------------------------------------------------------------
# r-z variance model of T3 / T5 on smeared helices
# ------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("region", ["barrel", "endcap"])
def test_rz_variance_model_matches_the_smearing(det, region):
    """chi2_rz per degree of freedom of truth-matched T3 (1 dof) and T5 (3 dof) whose anchors all lie
    in the barrel (z smeared by sigma_z) or all in the endcap (r smeared by sigma_r, seen in z as
    sigma_r |dz/ds|). The barrel mean sits just below 1 (the chi2 cuts truncate the tail); the endcap
    model is conservative (the circle through the smeared anchors absorbs part of their radial
    error) but of the right scale: a sigma_r without the slope factor (cot theta ~ 2.5-5.5 here)
    would give means of ~10 and more."""
    g = det.geom
    c3, c5 = [], []
    for seed in range(4):
        rng = np.random.default_rng(300 + seed)
        n = 250
        pt = gen._powerlaw_pt(rng, n, 0.8)
        if region == "barrel":
            eta = rng.uniform(-0.9, 0.9, n)
        else:
            eta = rng.choice([-1.0, 1.0], n) * rng.uniform(1.6, 2.4, n)
        ev = gen.simulate(g, rng, rng.choice([-1, 1], n), pt, rng.uniform(-math.pi, math.pi, n), eta,
                          np.zeros(n), rng.normal(0, 5, n), eff=1.0)
        r = oracle.run(det, ev)
        md = r["md"]
        hp = ev.hit_particle
        mdp = np.where(hp[md["hit_lo"]] == hp[md["hit_up"]], hp[md["hit_lo"]], -1)
        mdec = g.subdet[md["module"]] == gen.SUBDET_ENDCAP
        for tab, k, out in ((r["t3"], 3, c3), (r["t5"], 5, c5)):
            for i in range(len(tab["md0"])):
                ids = [tab[f"md{j}"][i] for j in range(k)]
                ps, ec = mdp[ids], mdec[ids]
                if ps[0] < 0 or not (ps == ps[0]).all():
                    continue
                if (region == "endcap" and ec.all()) or (region == "barrel" and not ec.any()):
                    out.append(tab["chi2_rz"][i])
    c3, c5 = np.array(c3), np.array(c5)
    assert c3.size > 1000 and c5.size > 100
    lo, hi = (0.8, 1.1) if region == "barrel" else (0.3, 1.2)
    assert lo <= c3.mean() <= hi, c3.mean()
    assert lo <= c5.mean() / 3 <= hi, c5.mean() / 3
