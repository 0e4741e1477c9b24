"""Seeded synthetic inputs for Line Segment Tracking: a toy outer-tracker geometry, the
module-connection map, the pixel-seed map and HL-LHC-like events.

This module is input generation only. It propagates ideal helices through a toy detector and
smears their crossings; it holds none of LST's selections (no Mini-Doublet, Segment, Triplet,
Quintuplet, pixel-object or Track-Candidate arithmetic). Both the CUDA path and the CPU oracle
consume what it produces, and neither is imported here.

Geometry (paper Sec. 2, "bi-layer pT modules" of the CMS outer tracker, Sec. 1):
  * barrel: 6 cylindrical layers, lower sensor radius r_L, upper sensor r_L + spacing, tiled by
    10 cm x 10 cm patches (n_phi = ceil(2 pi r_L / 10), 22 z-tiles over [-110, 110) cm);
  * endcap: 5 disks per side, lower sensor plane |z| = z_D, upper plane |z| = z_D + spacing,
    9 rings of 10 cm radial width from r = 23 cm to 110 cm, n_phi = ceil(2 pi r_mid / 10);
  * PS modules in barrel layers 1-3 and in rings with r_mid < 60 cm, 2S modules elsewhere.

The module map (paper Sec. 2.2) is derived from first principles: helices compatible with the pT
threshold are started at points of a module's lower sensor and the modules they reach on the next
layer are listed (with +-1 neighbours as tolerance).

All random numbers come from numpy's PCG64 seeded per event (seed = 1000 * config + event).
"""
from __future__ import annotations

import functools
import hashlib
import math
import os
from dataclasses import dataclass, field

import numpy as np

TWO_PI = 2.0 * math.pi

# pT[GeV] = K_B * R[cm] for a unit-charge helix in B = 3.8 T (0.003 * B).
K_B = 0.0114

BARREL_R = np.array([23.0, 36.0, 51.0, 68.0, 86.0, 110.0])
BARREL_SPACING = np.array([0.26, 0.26, 0.26, 0.40, 0.40, 0.40])
BARREL_NZ = 22
BARREL_ZHALF = 110.0
BARREL_ZTILE = 10.0

DISK_Z = np.array([131.0, 156.0, 185.0, 220.0, 262.0])
N_RINGS = 9
RING_R_LO = np.array([23.0 + 10.0 * m for m in range(N_RINGS)])
RING_R_HI = np.array([min(33.0 + 10.0 * m, 110.0) for m in range(N_RINGS)])
ENDCAP_R_MIN = 23.0
ENDCAP_R_MAX = 110.0
PS_RING_R_MAX = 60.0  # rings with r_mid below this are PS
# spacing by disk (1..5): PS / 2S
DISK_SPACING_PS = np.array([0.16, 0.16, 0.26, 0.26, 0.40])
DISK_SPACING_2S = np.array([0.18, 0.18, 0.40, 0.40, 0.40])

# outer envelope: a helix is followed until it leaves it (or completes one turn in xy)
R_OUT = 111.0
Z_OUT = 263.0

SUBDET_BARREL = 0
SUBDET_ENDCAP = 1
TYPE_PS = 0
TYPE_2S = 1

# hit resolution: 30 um in r-phi, 1 mm in z for barrel / r for endcap
SIGMA_RPHI = 0.003
SIGMA_Z = 0.1
SIGMA_R = 0.1

# pixel-map binning: eta in [-2.5, 2.5) by 0.05, phi in [0, 2pi) by 2pi/128, charge
PIX_NETA = 100
PIX_NPHI = 128
PIX_ETA_MIN = -2.5
PIX_ETA_W = 0.05
N_PIX_BINS = PIX_NETA * PIX_NPHI * 2

# lst_module record, laid out as the C-ABI struct (11 x 4 bytes)
MODULE_DTYPE = np.dtype([
    ("id", "<i4"), ("subdet", "<i4"), ("layer", "<i4"), ("side", "<i4"), ("type", "<i4"),
    ("surf", "<f4"), ("spacing", "<f4"), ("phi_lo", "<f4"), ("phi_hi", "<f4"),
    ("w_lo", "<f4"), ("w_hi", "<f4"),
])

# lst_pls record (pixel line segment seed), laid out as the C-ABI struct (48 bytes)
PLS_DTYPE = np.dtype([
    ("pt", "<f4"), ("eta", "<f4"), ("phi", "<f4"), ("x0", "<f4"), ("y0", "<f4"), ("z0", "<f4"),
    ("charge", "<i4"), ("pix_hit", "<i4", (4,)), ("_pad", "<i4"),
])


# --------------------------------------------------------------------------------------------
# geometry
# --------------------------------------------------------------------------------------------
@dataclass
class Geometry:
    barrel_only: bool
    n_mods: int
    subdet: np.ndarray
    layer: np.ndarray      # barrel layer 1..6 or disk 1..5
    side: np.ndarray       # 0 barrel, -1/+1 endcap
    mtype: np.ndarray      # TYPE_PS / TYPE_2S
    surf: np.ndarray       # r (barrel) or |z| (endcap) of the lower sensor
    spacing: np.ndarray
    phi_lo: np.ndarray
    phi_hi: np.ndarray
    w_lo: np.ndarray       # z range (barrel) or r range (endcap)
    w_hi: np.ndarray
    iphi: np.ndarray
    iw: np.ndarray         # z tile (barrel) or ring (endcap)
    nphi: np.ndarray
    barrel_base: np.ndarray            # [6] first module id of each barrel layer
    endcap_base: dict = field(default_factory=dict)  # (side, disk, ring) -> first module id

    @property
    def ec_base_arr(self) -> np.ndarray:
        a = np.full((2, 5, N_RINGS), -1, dtype=np.int64)
        for (side, d, m), v in self.endcap_base.items():
            a[(side + 1) // 2, d, m] = v
        return a

    def module_records(self) -> np.ndarray:
        rec = np.zeros(self.n_mods, dtype=MODULE_DTYPE)
        rec["id"] = np.arange(self.n_mods)
        rec["subdet"] = self.subdet
        rec["layer"] = self.layer
        rec["side"] = self.side
        rec["type"] = self.mtype
        rec["surf"] = self.surf
        rec["spacing"] = self.spacing
        rec["phi_lo"] = self.phi_lo
        rec["phi_hi"] = self.phi_hi
        rec["w_lo"] = self.w_lo
        rec["w_hi"] = self.w_hi
        return rec

    @property
    def n_sensors(self) -> int:
        return 2 * self.n_mods


def _barrel_nphi(L: int) -> int:
    return int(math.ceil(TWO_PI * BARREL_R[L] / 10.0))


def _ring_nphi(m: int) -> int:
    return int(math.ceil(TWO_PI * 0.5 * (RING_R_LO[m] + RING_R_HI[m]) / 10.0))


@functools.lru_cache(maxsize=4)
def make_geometry(barrel_only: bool = False) -> Geometry:
    cols = {k: [] for k in ("subdet", "layer", "side", "mtype", "surf", "spacing", "phi_lo",
                            "phi_hi", "w_lo", "w_hi", "iphi", "iw", "nphi")}
    barrel_base = np.zeros(6, dtype=np.int64)
    endcap_base = {}
    n = 0

    def add(**kw):
        for k, v in kw.items():
            cols[k].append(v)

    for L in range(6):
        barrel_base[L] = n
        nphi = _barrel_nphi(L)
        for j in range(BARREL_NZ):
            for i in range(nphi):
                add(subdet=SUBDET_BARREL, layer=L + 1, side=0, mtype=TYPE_PS if L < 3 else TYPE_2S,
                    surf=BARREL_R[L], spacing=BARREL_SPACING[L], phi_lo=TWO_PI * i / nphi,
                    phi_hi=TWO_PI * (i + 1) / nphi, w_lo=-BARREL_ZHALF + BARREL_ZTILE * j,
                    w_hi=-BARREL_ZHALF + BARREL_ZTILE * (j + 1), iphi=i, iw=j, nphi=nphi)
                n += 1
    if not barrel_only:
        for side in (-1, 1):
            for d in range(5):
                for m in range(N_RINGS):
                    endcap_base[(side, d, m)] = n
                    nphi = _ring_nphi(m)
                    rmid = 0.5 * (RING_R_LO[m] + RING_R_HI[m])
                    ps = rmid < PS_RING_R_MAX
                    sp = DISK_SPACING_PS[d] if ps else DISK_SPACING_2S[d]
                    for i in range(nphi):
                        add(subdet=SUBDET_ENDCAP, layer=d + 1, side=side,
                            mtype=TYPE_PS if ps else TYPE_2S, surf=DISK_Z[d], spacing=sp,
                            phi_lo=TWO_PI * i / nphi, phi_hi=TWO_PI * (i + 1) / nphi,
                            w_lo=RING_R_LO[m], w_hi=RING_R_HI[m], iphi=i, iw=m, nphi=nphi)
                        n += 1
    arr = {k: np.asarray(v) for k, v in cols.items()}
    return Geometry(
        barrel_only=barrel_only, n_mods=n,
        subdet=arr["subdet"].astype(np.int32), layer=arr["layer"].astype(np.int32),
        side=arr["side"].astype(np.int32), mtype=arr["mtype"].astype(np.int32),
        surf=arr["surf"].astype(np.float64), spacing=arr["spacing"].astype(np.float64),
        phi_lo=arr["phi_lo"], phi_hi=arr["phi_hi"], w_lo=arr["w_lo"], w_hi=arr["w_hi"],
        iphi=arr["iphi"].astype(np.int64), iw=arr["iw"].astype(np.int64),
        nphi=arr["nphi"].astype(np.int64), barrel_base=barrel_base, endcap_base=endcap_base)


# --------------------------------------------------------------------------------------------
# sensor surfaces
# --------------------------------------------------------------------------------------------
@dataclass(frozen=True)
class Surface:
    kind: str          # "cyl" or "plane"
    pos: float         # radius (cyl) or signed z (plane)
    layer: int         # barrel layer 0..5 or disk 0..4
    sensor: int        # 0 lower, 1 upper
    side: int          # 0 barrel, -1/+1 endcap
    r_lo: float = 0.0  # plane: accepted radial range (upper planes differ for PS and 2S rings)
    r_hi: float = 0.0


@functools.lru_cache(maxsize=4)
def surfaces(barrel_only: bool) -> tuple:
    out = []
    for L in range(6):
        out.append(Surface("cyl", float(BARREL_R[L]), L, 0, 0))
        out.append(Surface("cyl", float(BARREL_R[L] + BARREL_SPACING[L]), L, 1, 0))
    if not barrel_only:
        ps_r_hi = RING_R_HI[3]  # rings 0..3 are PS
        for side in (-1, 1):
            for d in range(5):
                z = float(DISK_Z[d])
                out.append(Surface("plane", side * z, d, 0, side, ENDCAP_R_MIN, ENDCAP_R_MAX))
                out.append(Surface("plane", side * (z + DISK_SPACING_PS[d]), d, 1, side,
                                   ENDCAP_R_MIN, float(ps_r_hi)))
                out.append(Surface("plane", side * (z + DISK_SPACING_2S[d]), d, 1, side,
                                   float(ps_r_hi), ENDCAP_R_MAX))
    return tuple(out)


# --------------------------------------------------------------------------------------------
# helix propagation (float64, vectorised over helices)
# --------------------------------------------------------------------------------------------
@dataclass
class Helices:
    """Helices parameterised at their point of closest approach to the z axis.

    q: charge (+-1); R: radius [cm]; phi0: direction at the PCA; cot: cot(theta); d0, z0.
    Position after turning angle psi >= 0 (B along +z, a positive charge turns clockwise):
        c = p0 + q R (sin phi0, -cos phi0),  p(psi) = c + q R (-sin(phi0 - q psi), cos(phi0 - q psi)),
        z(psi) = z0 + R psi cot.
    """
    q: np.ndarray
    R: np.ndarray
    phi0: np.ndarray
    cot: np.ndarray
    d0: np.ndarray
    z0: np.ndarray

    def __post_init__(self):
        self.x0 = -self.d0 * np.sin(self.phi0)
        self.y0 = self.d0 * np.cos(self.phi0)
        self.cx = self.x0 + self.q * self.R * np.sin(self.phi0)
        self.cy = self.y0 - self.q * self.R * np.cos(self.phi0)

    def __len__(self):
        return len(self.q)

    def position(self, psi):
        ang = self.phi0 - self.q * psi
        x = self.cx - self.q * self.R * np.sin(ang)
        y = self.cy + self.q * self.R * np.cos(ang)
        z = self.z0 + self.R * psi * self.cot
        return x, y, z


def cylinder_psi(h: Helices, rho: float):
    """Both turning angles in [0, 2 pi) at which the helix crosses the cylinder r = rho
    (NaN where it does not). Solves |c + q R u(psi)|^2 = rho^2 in closed form."""
    cn = np.hypot(h.cx, h.cy)
    gam = np.arctan2(h.cy, h.cx)
    with np.errstate(divide="ignore", invalid="ignore"):
        S = (rho * rho - cn * cn - h.R * h.R) / (2.0 * h.q * h.R * cn)
    ok = np.abs(S) <= 1.0
    A1 = np.arcsin(np.clip(S, -1.0, 1.0))
    A2 = math.pi - A1
    p1 = np.mod(h.q * (A1 - gam + h.phi0), TWO_PI)
    p2 = np.mod(h.q * (A2 - gam + h.phi0), TWO_PI)
    p1 = np.where(ok, p1, np.nan)
    p2 = np.where(ok, p2, np.nan)
    return p1, p2


def plane_psi(h: Helices, zp: float):
    with np.errstate(divide="ignore", invalid="ignore"):
        psi = (zp - h.z0) / (h.R * h.cot)
    return np.where(np.isfinite(psi) & (psi > 0.0), psi, np.nan)


def exit_psi(h: Helices):
    """Turning angle at which the helix leaves the tracker envelope, capped at one full turn."""
    p1, p2 = cylinder_psi(h, R_OUT)
    out = np.fmin(np.where(p1 > 1e-12, p1, np.nan), np.where(p2 > 1e-12, p2, np.nan))
    zexit = np.fmax(plane_psi(h, Z_OUT), plane_psi(h, -Z_OUT))
    out = np.fmin(out, zexit)
    return np.fmin(np.nan_to_num(out, nan=TWO_PI), TWO_PI)


def _wrap02pi(phi):
    return np.mod(phi, TWO_PI)


def locate_module(geom: Geometry, surf: Surface, x, y, z):
    """Module id (or -1 when outside every active patch) for crossing points on a surface."""
    phi = _wrap02pi(np.arctan2(y, x))
    if surf.kind == "cyl":
        L = surf.layer
        nphi = _barrel_nphi(L)
        j = np.floor((z + BARREL_ZHALF) / BARREL_ZTILE).astype(np.int64)
        i = np.minimum(np.floor(phi * nphi / TWO_PI).astype(np.int64), nphi - 1)
        ok = (z >= -BARREL_ZHALF) & (z < BARREL_ZHALF)
        mod = geom.barrel_base[L] + np.clip(j, 0, BARREL_NZ - 1) * nphi + i
        return np.where(ok, mod, -1)
    if geom.barrel_only:
        return np.full(np.shape(x), -1, dtype=np.int64)
    r = np.hypot(x, y)
    ok = (r >= surf.r_lo) & (r < surf.r_hi)
    m = np.clip(np.floor((r - ENDCAP_R_MIN) / 10.0).astype(np.int64), 0, N_RINGS - 1)
    out = np.full(np.shape(x), -1, dtype=np.int64)
    for ring in range(N_RINGS):
        sel = ok & (m == ring)
        if not np.any(sel):
            continue
        nphi = _ring_nphi(ring)
        i = np.minimum(np.floor(phi[sel] * nphi / TWO_PI).astype(np.int64), nphi - 1)
        out[sel] = geom.endcap_base[(surf.side, surf.layer, ring)] + i
    return out


def crossings(geom: Geometry, h: Helices, psi_min=None, lower_only=False):
    """All (helix index, surface index, psi, module, x, y, z) crossings of active sensors with
    psi in (psi_min, psi_exit]."""
    psi_max = exit_psi(h)
    lo = np.zeros(len(h)) if psi_min is None else psi_min
    rows = []
    for si, s in enumerate(surfaces(geom.barrel_only)):
        if lower_only and s.sensor != 0:
            continue
        if s.kind == "cyl":
            cands = cylinder_psi(h, s.pos)
        else:
            cands = (plane_psi(h, s.pos),)
        for psi in cands:
            ok = np.isfinite(psi) & (psi > lo + 1e-9) & (psi <= psi_max)
            idx = np.nonzero(ok)[0]
            if idx.size == 0:
                continue
            sub = Helices(h.q[idx], h.R[idx], h.phi0[idx], h.cot[idx], h.d0[idx], h.z0[idx])
            x, y, z = sub.position(psi[idx])
            if s.kind == "cyl":
                # put the point exactly on the cylinder (removes round-off of the closed form)
                rr = np.hypot(x, y)
                x, y = x * (s.pos / rr), y * (s.pos / rr)
            else:
                z = np.full_like(x, s.pos)
            mod = locate_module(geom, s, x, y, z)
            good = mod >= 0
            rows.append((idx[good], np.full(int(good.sum()), si), psi[idx][good], mod[good],
                         x[good], y[good], z[good]))
    if not rows:
        e = np.zeros(0)
        return (e.astype(np.int64),) * 2 + (e,) + (e.astype(np.int64),) + (e,) * 3
    cat = [np.concatenate([r[k] for r in rows]) for k in range(7)]
    order = np.lexsort((cat[2], cat[0]))
    return tuple(c[order] for c in cat)


# --------------------------------------------------------------------------------------------
# module map (paper Sec. 2.2) and pixel map
# --------------------------------------------------------------------------------------------
def _neighbours(geom: Geometry, mods: np.ndarray) -> np.ndarray:
    """Each module with its +-1 neighbours in phi and in z-tile (barrel) or ring (endcap)."""
    out = []
    for dm in (-1, 0, 1):
        for di in (-1, 0, 1):
            res = np.full(mods.shape, -1, dtype=np.int64)
            b = geom.subdet[mods] == SUBDET_BARREL
            if np.any(b):
                mb = mods[b]
                L = geom.layer[mb] - 1
                nphi = geom.nphi[mb]
                j = geom.iw[mb] + dm
                i = np.mod(geom.iphi[mb] + di, nphi)
                okj = (j >= 0) & (j < BARREL_NZ)
                res[b] = np.where(okj, geom.barrel_base[L] + np.clip(j, 0, BARREL_NZ - 1) * nphi + i, -1)
            e = ~b
            if np.any(e):
                me = mods[e]
                ring = geom.iw[me] + dm
                phic = 0.5 * (geom.phi_lo[me] + geom.phi_hi[me])
                vals = np.full(me.shape, -1, dtype=np.int64)
                for r in range(N_RINGS):
                    sel = ring == r
                    if not np.any(sel):
                        continue
                    mm = me[sel]
                    nphi = _ring_nphi(r)
                    i0 = np.floor(phic[sel] * nphi / TWO_PI).astype(np.int64)
                    i = np.mod(i0 + di, nphi)
                    base = geom.ec_base_arr[(geom.side[mm] + 1) // 2, geom.layer[mm] - 1, r]
                    vals[sel] = base + i
                res[e] = vals
            out.append(res)
    # adjacent rings have different phi tilings: also take every module of ring +-1 whose
    # phi range overlaps this module's phi range (handled by the +-1 around the centre above,
    # since ring phi widths differ by less than a factor of two between adjacent rings)
    allm = np.stack(out, axis=1)
    return allm


def _csr(pairs_src: np.ndarray, pairs_dst: np.ndarray, n_src: int):
    key = np.unique(pairs_src.astype(np.int64) * (1 << 32) + pairs_dst.astype(np.int64))
    src = (key >> 32).astype(np.int64)
    dst = (key & 0xFFFFFFFF).astype(np.int32)
    off = np.zeros(n_src + 1, dtype=np.int32)
    np.add.at(off, src + 1, 1)
    return np.cumsum(off).astype(np.int32), dst


MAP_PTS = (None, 1.5, 3.0, 10.0, 100.0)   # None -> pT threshold
Z_LUM = 15.0


def _helix_through(q, pt, z0, px, py, pz):
    """d0 = 0 helix from (0, 0, z0) through point P (the shorter arc); returns (Helices, psi_P).
    Points beyond the helix's reach (|P| > 2R) are marked with psi_P = NaN."""
    R = pt / K_B
    rho = np.hypot(px, py)
    s = rho / (2.0 * R)
    ok = s <= 1.0
    alpha = np.arcsin(np.clip(s, 0.0, 1.0))
    phiP = np.arctan2(py, px)
    phi0 = phiP + q * alpha
    psiP = 2.0 * alpha
    with np.errstate(divide="ignore", invalid="ignore"):
        cot = (pz - z0) / (R * psiP)
    h = Helices(q.astype(np.float64), R, phi0, cot, np.zeros_like(R), z0)
    return h, np.where(ok, psiP, np.nan)


def build_module_map(geom: Geometry, pt_thr: float = 0.8, grid: int = 9, chunk: int = 1_500_000):
    """Module-connection map as CSR (offsets [n_mods+1], targets).

    For each module A, helices with pT in {pT_thr, 1.5, 3, 10, 100} GeV, both charges and
    z0 in {-z_lum, 0, +z_lum} are passed through a grid x grid set of points of A's lower sensor
    (edges included). The module each reaches on the next lower-sensor surface outward is listed
    with its +-1 phi and z/ring neighbours."""
    n = geom.n_mods
    u = np.linspace(0.0, 1.0, grid)
    uu, vv = np.meshgrid(u, u, indexing="ij")
    uu, vv = uu.ravel(), vv.ravel()
    mod = np.repeat(np.arange(n), grid * grid)
    fu = np.tile(uu, n)
    fv = np.tile(vv, n)
    phi = geom.phi_lo[mod] + fu * (geom.phi_hi[mod] - geom.phi_lo[mod])
    w = geom.w_lo[mod] + fv * (geom.w_hi[mod] - geom.w_lo[mod])
    barrel = geom.subdet[mod] == SUBDET_BARREL
    rho = np.where(barrel, geom.surf[mod], w)
    px, py = rho * np.cos(phi), rho * np.sin(phi)
    pz = np.where(barrel, w, geom.side[mod] * geom.surf[mod])

    combos = [(q, pt, z0) for q in (-1, 1) for pt in MAP_PTS for z0 in (-Z_LUM, 0.0, Z_LUM)]
    src_all, dst_all = [], []
    lower_surfs = [(si, s) for si, s in enumerate(surfaces(geom.barrel_only)) if s.sensor == 0]
    npts = mod.size
    for q, pt, z0 in combos:
        ptv = pt_thr if pt is None else pt
        for c0 in range(0, npts, chunk):
            sl = slice(c0, min(npts, c0 + chunk))
            m_a = mod[sl]
            k = m_a.size
            h, psiP = _helix_through(np.full(k, q), np.full(k, ptv), np.full(k, z0),
                                     px[sl], py[sl], pz[sl])
            psi_max = exit_psi(h)
            best = np.full(k, np.inf)
            best_mod = np.full(k, -1, dtype=np.int64)
            a_barrel = geom.subdet[m_a] == SUBDET_BARREL
            a_layer = geom.layer[m_a] - 1
            a_side = geom.side[m_a]
            for si, s in lower_surfs:
                if s.kind == "cyl":
                    elig = a_barrel & (s.layer > a_layer)
                    cands = cylinder_psi(h, s.pos)
                else:
                    # outward: a disk further out on the side the helix is moving towards
                    elig = np.where(a_barrel, np.sign(h.cot) == s.side,
                                    (a_side == s.side) & (s.layer > a_layer))
                    cands = (plane_psi(h, s.pos),)
                for psi in cands:
                    ok = elig & np.isfinite(psi) & np.isfinite(psiP) & (psi > psiP + 1e-9) & \
                        (psi <= psi_max) & (psi < best)
                    idx = np.nonzero(ok)[0]
                    if idx.size == 0:
                        continue
                    sub = Helices(h.q[idx], h.R[idx], h.phi0[idx], h.cot[idx], h.d0[idx], h.z0[idx])
                    x, y, z = sub.position(psi[idx])
                    if s.kind == "plane":
                        z = np.full_like(x, s.pos)
                    mb = locate_module(geom, s, x, y, z)
                    good = mb >= 0
                    best[idx[good]] = psi[idx][good]
                    best_mod[idx[good]] = mb[good]
            hit = best_mod >= 0
            if np.any(hit):
                pairs = np.unique(m_a[hit] * (1 << 32) + best_mod[hit])
                src_all.append(pairs >> 32)
                dst_all.append(pairs & 0xFFFFFFFF)
    src = np.concatenate(src_all)
    dst = np.concatenate(dst_all)
    key = np.unique(src * (1 << 32) + dst)
    src, dst = key >> 32, key & 0xFFFFFFFF
    nb = _neighbours(geom, dst)
    src_rep = np.repeat(src, nb.shape[1])
    nbf = nb.ravel()
    keep = nbf >= 0
    return _csr(src_rep[keep], nbf[keep], n)


PIX_PTS = (None, 1.0, 1.5, 2.5, 5.0, 100.0)   # None -> pT threshold


def pixel_bin_of(eta, phi, charge):
    """Pixel-map bin of a seed: (floor(20 eta + 50), floor(wrap_[0,2pi)(phi) * 64 / pi), charge).
    Returns -1 for eta outside [-2.5, 2.5)."""
    ie = np.floor(np.asarray(eta, np.float64) * 20.0 + 50.0).astype(np.int64)
    ph = np.asarray(phi, np.float64)
    ph = np.where(ph < 0.0, ph + TWO_PI, ph)
    ip = np.floor(ph * (64.0 / math.pi)).astype(np.int64)
    ip = np.clip(ip, 0, PIX_NPHI - 1)
    iq = (np.asarray(charge) > 0).astype(np.int64)
    b = (ie * PIX_NPHI + ip) * 2 + iq
    return np.where((ie >= 0) & (ie < PIX_NETA), b, -1)


def build_pixel_map(geom: Geometry, pt_thr: float = 0.8, chunk: int = 1_000_000):
    """Pixel map as CSR over N_PIX_BINS bins: for each (eta, phi, charge) bin, the modules on the
    first three lower-sensor surfaces crossed by d0 = 0 helices started from the bin's corners and
    centre, with pT in {pT_thr, 1, 1.5, 2.5, 5, 100} GeV and z0 in {-z_lum, 0, z_lum}, each with
    its +-1 neighbours."""
    fr = np.array([0.0, 0.5, 1.0])
    ie, ip, iq, fe, fp, ipt, iz = np.meshgrid(np.arange(PIX_NETA), np.arange(PIX_NPHI), np.arange(2),
                                             fr, fr, np.arange(len(PIX_PTS)), np.arange(3),
                                             indexing="ij")
    ie, ip, iq, fe, fp, ipt, iz = (a.ravel() for a in (ie, ip, iq, fe, fp, ipt, iz))
    bins = (ie * PIX_NPHI + ip) * 2 + iq
    eta = PIX_ETA_MIN + PIX_ETA_W * (ie + fe)
    phi = (TWO_PI / PIX_NPHI) * (ip + fp)
    q = np.where(iq == 1, 1.0, -1.0)
    pts = np.array([pt_thr if p is None else p for p in PIX_PTS])
    pt = pts[ipt]
    z0 = np.array([-Z_LUM, 0.0, Z_LUM])[iz]
    src_all, dst_all = [], []
    for c0 in range(0, bins.size, chunk):
        sl = slice(c0, min(bins.size, c0 + chunk))
        h = Helices(q[sl], pt[sl] / K_B, phi[sl], np.sinh(eta[sl]), np.zeros(bins[sl].size), z0[sl])
        hi, si, psi, mods, *_ = crossings(geom, h, lower_only=True)
        if hi.size == 0:
            continue
        surf_layer_key = np.array([(s.kind == "plane") * 10 + s.layer for s in surfaces(geom.barrel_only)])
        lk = surf_layer_key[si]
        # rank of each crossing's layer among the distinct layers this helix crossed (in psi order)
        order = np.lexsort((psi, hi))
        hi, lk, mods = hi[order], lk[order], mods[order]
        first = np.ones(hi.size, dtype=bool)
        first[1:] = (hi[1:] != hi[:-1]) | (lk[1:] != lk[:-1])
        newhel = np.ones(hi.size, dtype=bool)
        newhel[1:] = hi[1:] != hi[:-1]
        grp = np.cumsum(newhel) - 1
        cnt = np.cumsum(first)
        start = cnt[np.nonzero(newhel)[0]][grp]
        rank = cnt - start  # 0-based layer rank
        keep = rank < 3
        b = bins[sl][hi[keep]]
        pairs = np.unique(b * (1 << 32) + mods[keep])
        src_all.append(pairs >> 32)
        dst_all.append(pairs & 0xFFFFFFFF)
    src = np.concatenate(src_all)
    dst = np.concatenate(dst_all)
    key = np.unique(src * (1 << 32) + dst)
    src, dst = key >> 32, key & 0xFFFFFFFF
    nb = _neighbours(geom, dst)
    src_rep = np.repeat(src, nb.shape[1])
    nbf = nb.ravel()
    keep = nbf >= 0
    return _csr(src_rep[keep], nbf[keep], N_PIX_BINS)


@dataclass
class Detector:
    """Geometry plus its module map and pixel map for one pT threshold."""
    geom: Geometry
    pt_thr: float
    conn_off: np.ndarray
    conn_tgt: np.ndarray
    pix_off: np.ndarray
    pix_tgt: np.ndarray

    @property
    def n_mods(self):
        return self.geom.n_mods


_CACHE_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_cache")


def _source_digest() -> str:
    with open(os.path.abspath(__file__), "rb") as f:
        return hashlib.sha1(f.read()).hexdigest()[:16]


@functools.lru_cache(maxsize=4)
def make_detector(barrel_only: bool = False, pt_thr: float = 0.8) -> Detector:
    """Geometry + module map + pixel map. The maps take tens of seconds to build, so they are
    kept in an on-disk cache next to this file, keyed by this file's content."""
    geom = make_geometry(barrel_only)
    path = os.path.join(_CACHE_DIR, f"det_b{int(barrel_only)}_pt{pt_thr:.3f}_{_source_digest()}.npz")
    if os.path.exists(path):
        try:
            with np.load(path) as d:
                return Detector(geom, pt_thr, d["co"], d["ct"], d["po"], d["pt"])
        except Exception:  # a truncated or foreign file: rebuild
            pass
    co, ct = build_module_map(geom, pt_thr)
    if barrel_only:
        po = np.zeros(N_PIX_BINS + 1, dtype=np.int32)
        pt = np.zeros(0, dtype=np.int32)
    else:
        po, pt = build_pixel_map(geom, pt_thr)
    try:
        os.makedirs(_CACHE_DIR, exist_ok=True)
        tmp = f"{path}.{os.getpid()}.tmp.npz"
        np.savez(tmp, co=co, ct=ct, po=po, pt=pt)
        os.replace(tmp, path)
    except OSError:
        pass
    return Detector(geom, pt_thr, co, ct, po, pt)


# --------------------------------------------------------------------------------------------
# events
# --------------------------------------------------------------------------------------------
@dataclass
class Event:
    x: np.ndarray          # float32 [n_hits]
    y: np.ndarray
    z: np.ndarray
    sensor: np.ndarray     # int32 [n_hits], 2 * module + (0 lower | 1 upper)
    pls: np.ndarray        # PLS_DTYPE [n_pls]
    hit_particle: np.ndarray   # truth: particle index per hit, -1 for noise
    pls_particle: np.ndarray   # truth: particle index per pLS
    particles: dict            # truth parameters per particle
    pu: float = 0.0

    @property
    def n_hits(self):
        return int(self.x.size)

    @property
    def n_pls(self):
        return int(self.pls.size)


def _powerlaw_pt(rng, n, pt_min):
    # dN/dpT ~ pT^-3 above pt_min: CDF 1 - (pt_min/pT)^2
    return pt_min / np.sqrt(1.0 - rng.random(n))


def simulate(geom: Geometry, rng: np.random.Generator, q, pt, phi0, eta, d0, z0, *, eff=0.99,
             noise_frac=0.0, clustered_noise=False, pls_min_pt=None, shuffle=True) -> Event:
    """Propagate helices through the detector, smear, add noise and build pixel seeds."""
    n = q.size
    h = Helices(q.astype(np.float64), pt / K_B, phi0, np.sinh(eta), d0, z0)
    pi_, si_, psi, mod, x, y, z = crossings(geom, h)
    surfs = surfaces(geom.barrel_only)
    sens = np.array([s.sensor for s in surfs])[si_]
    kind_cyl = np.array([s.kind == "cyl" for s in surfs])[si_]
    keep = rng.random(pi_.size) < eff
    pi_, sens, kind_cyl, mod, x, y, z = (a[keep] for a in (pi_, sens, kind_cyl, mod, x, y, z))
    r = np.hypot(x, y)
    phi = np.arctan2(y, x)
    g_rphi = rng.standard_normal(r.size) * SIGMA_RPHI
    g_w = rng.standard_normal(r.size)
    rs = np.where(kind_cyl, r, r + g_w * SIGMA_R)
    phis = phi + g_rphi / r
    zs = np.where(kind_cyl, z + g_w * SIGMA_Z, z)
    xs, ys = rs * np.cos(phis), rs * np.sin(phis)
    sensor = 2 * mod + sens
    hit_particle = pi_.astype(np.int64)

    n_sig = xs.size
    n_noise = int(round(noise_frac / (1.0 - noise_frac) * n_sig)) if noise_frac > 0 else 0
    if n_noise:
        if clustered_noise and n_sig:
            # noise clustered within +-2 cm (on-sensor r-phi and z/r) of particle hits
            src = rng.integers(0, n_sig, n_noise)
            du = rng.uniform(-2.0, 2.0, n_noise)
            dw = rng.uniform(-2.0, 2.0, n_noise)
            nmod = sensor[src] // 2
            nsens = sensor[src] % 2
            barrel = geom.subdet[nmod] == SUBDET_BARREL
            rr = np.hypot(xs[src], ys[src])
            ph = np.arctan2(ys[src], xs[src]) + du / rr
            rn = np.where(barrel, rr, rr + dw)
            zn = np.where(barrel, zs[src] + dw, zs[src])
            phw = _wrap02pi(ph)
            inside = (phw >= geom.phi_lo[nmod]) & (phw < geom.phi_hi[nmod])
            inside &= np.where(barrel, (zn >= geom.w_lo[nmod]) & (zn < geom.w_hi[nmod]),
                               (rn >= geom.w_lo[nmod]) & (rn < geom.w_hi[nmod]))
            nx, ny, nz = rn * np.cos(ph), rn * np.sin(ph), zn
            nsensor = 2 * nmod + nsens
            nx, ny, nz, nsensor = nx[inside], ny[inside], nz[inside], nsensor[inside]
        else:
            nmod = rng.integers(0, geom.n_mods, n_noise)
            nsens = rng.integers(0, 2, n_noise)
            barrel = geom.subdet[nmod] == SUBDET_BARREL
            ph = geom.phi_lo[nmod] + rng.random(n_noise) * (geom.phi_hi[nmod] - geom.phi_lo[nmod])
            wv = geom.w_lo[nmod] + rng.random(n_noise) * (geom.w_hi[nmod] - geom.w_lo[nmod])
            sp = geom.spacing[nmod] * nsens
            rn = np.where(barrel, geom.surf[nmod] + sp, wv)
            nz = np.where(barrel, wv, geom.side[nmod] * (geom.surf[nmod] + sp))
            nx, ny = rn * np.cos(ph), rn * np.sin(ph)
            nsensor = 2 * nmod + nsens
        xs = np.concatenate([xs, nx])
        ys = np.concatenate([ys, ny])
        zs = np.concatenate([zs, nz])
        sensor = np.concatenate([sensor, nsensor])
        hit_particle = np.concatenate([hit_particle, np.full(nx.size, -1)])

    if shuffle:
        perm = rng.permutation(xs.size)
        xs, ys, zs, sensor, hit_particle = (a[perm] for a in (xs, ys, zs, sensor, hit_particle))
    n_hits = xs.size

    # pixel line segments: one per particle above pls_min_pt, parameters smeared
    if pls_min_pt is not None:
        sel = np.nonzero(pt > pls_min_pt)[0]
        m = sel.size
        theta = 2.0 * np.arctan(np.exp(-eta[sel]))
        pt_s = pt[sel] * (1.0 + 0.01 * rng.standard_normal(m))
        phi_s = phi0[sel] + 1e-3 * rng.standard_normal(m)
        th_s = theta + 1e-3 * rng.standard_normal(m)
        eta_s = -np.log(np.tan(0.5 * th_s))
        pls = np.zeros(m, dtype=PLS_DTYPE)
        pls["pt"] = pt_s
        pls["eta"] = eta_s
        pls["phi"] = np.arctan2(np.sin(phi_s), np.cos(phi_s))
        pls["x0"] = -d0[sel] * np.sin(phi0[sel])
        pls["y0"] = d0[sel] * np.cos(phi0[sel])
        pls["z0"] = z0[sel]
        pls["charge"] = q[sel]
        pls["pix_hit"] = n_hits + 4 * np.arange(m)[:, None] + np.arange(4)[None, :]
        pls_particle = sel.astype(np.int32)
    else:
        pls = np.zeros(0, dtype=PLS_DTYPE)
        pls_particle = np.zeros(0, dtype=np.int32)

    return Event(
        x=xs.astype(np.float32), y=ys.astype(np.float32), z=zs.astype(np.float32),
        sensor=sensor.astype(np.int32), pls=pls, hit_particle=hit_particle.astype(np.int32),
        pls_particle=pls_particle,
        particles=dict(q=q, pt=pt, phi0=phi0, eta=eta, d0=d0, z0=z0))


def single_helix_event(geom: Geometry, q: int, pt: float, eta: float, phi0: float = 0.3,
                       z0: float = 0.0, d0: float = 0.0, smear: bool = False, seed: int = 0) -> Event:
    """One noise-free helix (optionally smeared), every crossing kept: for closed-form tests."""
    rng = np.random.default_rng(seed)
    ev = simulate(geom, rng, np.array([q]), np.array([pt]), np.array([phi0]), np.array([eta]),
                  np.array([d0]), np.array([z0]), eff=1.0, shuffle=False)
    if not smear:
        h = Helices(np.array([float(q)]), np.array([pt / K_B]), np.array([phi0]),
                    np.array([math.sinh(eta)]), np.array([d0]), np.array([z0]))
        _, _, _, mod, x, y, z = crossings(geom, h)
        ev.x, ev.y, ev.z = x.astype(np.float32), y.astype(np.float32), z.astype(np.float32)
    return ev


def config_event(config: int, event: int = 0, pu: float | None = None) -> tuple:
    """(Detector, Event) for one event of a benchmark configuration (seed = 1000*config + event).

    1: toy barrel, 200 helices, pT log-uniform 1-10 GeV, |eta| < 1, no noise, no seeds.
    2: full tracker, PU200: 30 helices per unit pile-up, dN/dpT ~ pT^-3 above 0.8 GeV,
       |eta| < 2.4, z0 ~ N(0, 5), d0 ~ N(0, 0.01), 3% uniform noise, 99% efficiency, one pLS per
       particle with pT > 0.8 GeV.
    3: as 2 with PU ~ U[140, 250].
    4: PU300, pT threshold 0.6 GeV, 20% loopers with pT ~ U[0.6, 0.9], 5% clustered noise.
    5: as 2 with PU ~ U[50, 300].
    """
    seed = 1000 * config + event
    rng = np.random.default_rng(seed)
    if config == 1:
        det = make_detector(barrel_only=True, pt_thr=0.8)
        n = 200
        pt = np.exp(rng.uniform(math.log(1.0), math.log(10.0), n))
        eta = rng.uniform(-1.0, 1.0, n)
        phi0 = rng.uniform(-math.pi, math.pi, n)
        z0 = rng.normal(0.0, 5.0, n)
        q = rng.choice([-1, 1], n)
        ev = simulate(det.geom, rng, q, pt, phi0, eta, np.zeros(n), z0, eff=1.0)
        return det, ev
    if config in (2, 3, 5):
        det = make_detector(barrel_only=False, pt_thr=0.8)
        if pu is None:
            pu = {2: 200.0, 3: rng.uniform(140.0, 250.0), 5: rng.uniform(50.0, 300.0)}[config]
        n = int(round(30 * pu))
        pt = _powerlaw_pt(rng, n, 0.8)
        eta = rng.uniform(-2.4, 2.4, n)
        phi0 = rng.uniform(-math.pi, math.pi, n)
        z0 = rng.normal(0.0, 5.0, n)
        d0 = rng.normal(0.0, 0.01, n)
        q = rng.choice([-1, 1], n)
        ev = simulate(det.geom, rng, q, pt, phi0, eta, d0, z0, eff=0.99, noise_frac=0.03,
                      pls_min_pt=0.8)
        ev.pu = pu
        return det, ev
    if config == 4:
        det = make_detector(barrel_only=False, pt_thr=0.6)
        pu = 300.0 if pu is None else pu
        n = int(round(30 * pu))
        looper = rng.random(n) < 0.2
        pt = np.where(looper, rng.uniform(0.6, 0.9, n), _powerlaw_pt(rng, n, 0.6))
        eta = rng.uniform(-2.4, 2.4, n)
        phi0 = rng.uniform(-math.pi, math.pi, n)
        z0 = rng.normal(0.0, 5.0, n)
        d0 = rng.normal(0.0, 0.01, n)
        q = rng.choice([-1, 1], n)
        ev = simulate(det.geom, rng, q, pt, phi0, eta, d0, z0, eff=0.99, noise_frac=0.05,
                      clustered_noise=True, pls_min_pt=0.6)
        ev.pu = pu
        return det, ev
    raise ValueError(f"unknown config {config}")


def small_event(n_particles: int, seed: int, barrel_only=False, noise_frac=0.03, pt_min=0.8,
                eta_max=2.4, with_pls=True) -> tuple:
    """A config-2-shaped event with a chosen particle count (parity tests at small sizes)."""
    det = make_detector(barrel_only=barrel_only, pt_thr=0.8)
    rng = np.random.default_rng(seed)
    n = n_particles
    pt = _powerlaw_pt(rng, n, pt_min)
    eta = rng.uniform(-eta_max, eta_max, n)
    phi0 = rng.uniform(-math.pi, math.pi, n)
    z0 = rng.normal(0.0, 5.0, n)
    d0 = rng.normal(0.0, 0.01, n)
    q = rng.choice([-1, 1], n)
    ev = simulate(det.geom, rng, q, pt, phi0, eta, d0, z0, eff=0.99, noise_frac=noise_frac,
                  pls_min_pt=0.8 if with_pls else None)
    return det, ev
