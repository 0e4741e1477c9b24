"""Pins of the synthetic-input generator: helix crossings against numeric root finding, the toy
geometry's module counts, and completeness of the module map and pixel map (paper Sec. 2.2: the
map lists every module reachable by a helix above the pT threshold)."""
import math

import numpy as np
import pytest
from scipy.optimize import brentq

from paper_2207_08207_gb300 import gen


def test_geometry_counts():
    g = gen.make_geometry(False)
    # barrel: sum ceil(2 pi r / 10) x 22 ; endcap: 388 modules per disk x 10 disks
    assert int((g.subdet == 0).sum()) == 5258
    assert int((g.subdet == 1).sum()) == 3880
    assert g.n_mods == 9138
    assert gen.make_geometry(True).n_mods == 5258


def _radius(h, i, psi):
    x, y, _ = gen.Helices(h.q[i:i + 1], h.R[i:i + 1], h.phi0[i:i + 1], h.cot[i:i + 1],
                          h.d0[i:i + 1], h.z0[i:i + 1]).position(np.array([psi]))
    return float(np.hypot(x, y)[0])


def test_cylinder_crossing_matches_root_finding():
    rng = np.random.default_rng(5)
    n = 200
    q = rng.choice([-1.0, 1.0], n)
    pt = rng.uniform(0.6, 20.0, n)
    h = gen.Helices(q, pt / gen.K_B, rng.uniform(-math.pi, math.pi, n), rng.uniform(-3, 3, n),
                    rng.normal(0, 0.5, n), rng.normal(0, 5, n))
    for rho in (23.0, 51.0, 86.3):
        p1, p2 = gen.cylinder_psi(h, rho)
        for i in range(n):
            f = lambda s: _radius(h, i, s) - rho
            for p in (p1[i], p2[i]):
                if np.isfinite(p):
                    assert abs(f(p)) < 1e-9
            # the first crossing from root finding on a fine grid agrees with the closed form
            grid = np.linspace(1e-9, 2 * math.pi - 1e-9, 4001)
            vals = np.array([f(s) for s in grid])
            sgn = np.nonzero(np.sign(vals[1:]) != np.sign(vals[:-1]))[0]
            roots = [brentq(f, grid[k], grid[k + 1], xtol=1e-14) for k in sgn]
            mine = sorted(p for p in (p1[i], p2[i]) if np.isfinite(p) and p > 1e-6)
            assert len(roots) == len(mine)
            for a, b in zip(roots, mine):
                assert abs(a - b) < 1e-8


def test_plane_crossing():
    h = gen.Helices(np.array([1.0]), np.array([100.0]), np.array([0.3]), np.array([1.5]),
                    np.array([0.0]), np.array([2.0]))
    psi = gen.plane_psi(h, 131.0)
    _, _, z = h.position(psi)
    assert abs(z[0] - 131.0) < 1e-12


def _lower_crossings(det, q, pt, phi0, eta, z0):
    h = gen.Helices(q, pt / gen.K_B, phi0, np.sinh(eta), np.zeros_like(q), z0)
    hi, si, psi, mod, x, y, z = gen.crossings(det.geom, h, lower_only=True)
    surfs = gen.surfaces(det.geom.barrel_only)
    layer_key = np.array([(s.kind == "plane") * 10 + s.layer for s in surfs])[si]
    return hi, psi, mod, layer_key


@pytest.mark.parametrize("barrel_only", [True, False])
def test_module_map_complete(barrel_only):
    det = gen.make_detector(barrel_only=barrel_only, pt_thr=0.8)
    rng = np.random.default_rng(11)
    n = 10000
    q = rng.choice([-1.0, 1.0], n)
    pt = 0.8 / np.sqrt(1.0 - rng.random(n))
    eta = rng.uniform(-1.0 if barrel_only else -2.4, 1.0 if barrel_only else 2.4, n)
    z0 = rng.uniform(-15.0, 15.0, n)
    hi, psi, mod, lk = _lower_crossings(det, q, pt, rng.uniform(-math.pi, math.pi, n), eta, z0)
    co, ct = det.conn_off, det.conn_tgt
    missing = 0
    pairs = 0
    for k in range(len(hi) - 1):
        if hi[k] != hi[k + 1] or lk[k] == lk[k + 1]:
            continue
        a, b = mod[k], mod[k + 1]
        pairs += 1
        if b not in ct[co[a]:co[a + 1]]:
            missing += 1
    assert pairs > 10000
    assert missing == 0


def test_pixel_map_complete():
    det = gen.make_detector(barrel_only=False, pt_thr=0.8)
    rng = np.random.default_rng(12)
    n = 5000
    q = rng.choice([-1.0, 1.0], n)
    pt = 0.8 / np.sqrt(1.0 - rng.random(n))
    eta = rng.uniform(-2.4, 2.4, n)
    phi0 = rng.uniform(-math.pi, math.pi, n)
    z0 = rng.uniform(-15.0, 15.0, n)
    hi, psi, mod, lk = _lower_crossings(det, q, pt, phi0, eta, z0)
    bins = gen.pixel_bin_of(eta, phi0, q)
    po, pt_ = det.pix_off, det.pix_tgt
    checked = missing = 0
    for i in range(n):
        sel = np.nonzero(hi == i)[0]
        layers = []
        for k in sel:
            if lk[k] not in layers:
                layers.append(lk[k])
            if len(layers) > 3:
                break
            b = bins[i]
            checked += 1
            if mod[k] not in pt_[po[b]:po[b + 1]]:
                missing += 1
    assert checked > 10000
    assert missing == 0
