"""Physics performance of track candidates on simulation truth (paper Sec. 3).

A track candidate (TC) is matched to a simulated particle when at least 75 % of its hits belong to
that particle. Efficiency is the fraction of simulated particles (in a pT or eta bin) that have a
matched TC; eta bins use particles above 0.9 GeV. The fake rate is the fraction of TCs matched to
no particle; the duplicate rate is the fraction of TCs whose particle is matched by two or more
TCs (all of them count as duplicates).

Host-side analysis of the chain's output: it reads TC rows (type, hit ids) and the generator's
truth (the particle of every hit and of every pixel seed) and is not part of the tracking path.
It works the same on the CUDA library's TCs and on the oracle's.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

MATCH_FRACTION = 0.75
PT_BINS = np.array([0.4, 0.5, 0.6, 0.7, 0.75, 0.8, 0.85, 0.9, 1.0, 1.2, 1.5, 2.0, 3.0, 5.0, 10.0, 100.0])
ETA_BINS = np.linspace(-2.4, 2.4, 13)
ETA_PT_MIN = 0.9
TC_TYPE_NAMES = ("pT5", "pT3", "T5", "pLS")


def hit_truth(ev) -> np.ndarray:
    """Particle of every hit id a TC row can hold, as a lookup array (-1: noise or unknown):
    outer-tracker hits by input index, pixel hits by the ids of the seed they belong to."""
    pix = np.asarray(ev.pls["pix_hit"], dtype=np.int64).reshape(-1) if ev.n_pls else np.zeros(0, np.int64)
    n = max(ev.n_hits, int(pix.max()) + 1 if pix.size else 0)
    lut = np.full(n + 1, -1, dtype=np.int64)
    lut[: ev.n_hits] = ev.hit_particle
    if pix.size:
        lut[pix] = np.repeat(np.asarray(ev.pls_particle, dtype=np.int64), 4)
    return lut


def match_tcs(tc_hits, lut: np.ndarray, fraction: float = MATCH_FRACTION) -> np.ndarray:
    """Matched particle of each TC (-1: fake). tc_hits: [n, 14] hit ids, -1 padded; lut: particle of
    each hit id (hit_truth)."""
    h = np.asarray(tc_hits, dtype=np.int64).reshape(-1, 14)
    valid = h >= 0
    part = np.where(valid, lut[np.clip(h, 0, lut.size - 1)], -1)
    part = np.where(valid & (h < lut.size), part, -1)
    n_hits = valid.sum(axis=1)
    # for each hit, how many hits of the row share its particle; the row's best particle
    same = (part[:, :, None] == part[:, None, :]) & (part[:, :, None] >= 0)
    cnt = same.sum(axis=2)
    k = np.argmax(cnt, axis=1)
    best = part[np.arange(h.shape[0]), k]
    ok = (best >= 0) & (cnt[np.arange(h.shape[0]), k] >= fraction * n_hits) & (n_hits > 0)
    return np.where(ok, best, -1)


@dataclass
class Counts:
    """Accumulated counts over events (numerators and denominators of the rates)."""
    eff_pt_num: np.ndarray = field(default_factory=lambda: np.zeros(len(PT_BINS) - 1, np.int64))
    eff_pt_den: np.ndarray = field(default_factory=lambda: np.zeros(len(PT_BINS) - 1, np.int64))
    eff_eta_num: np.ndarray = field(default_factory=lambda: np.zeros(len(ETA_BINS) - 1, np.int64))
    eff_eta_den: np.ndarray = field(default_factory=lambda: np.zeros(len(ETA_BINS) - 1, np.int64))
    eff_pt_by_type: np.ndarray = field(default_factory=lambda: np.zeros((4, len(PT_BINS) - 1), np.int64))
    n_tc: int = 0
    n_fake: int = 0
    n_dup: int = 0
    n_tc_type: np.ndarray = field(default_factory=lambda: np.zeros(4, np.int64))
    n_fake_type: np.ndarray = field(default_factory=lambda: np.zeros(4, np.int64))
    n_dup_type: np.ndarray = field(default_factory=lambda: np.zeros(4, np.int64))

    def add(self, ev, tc_type, tc_hits):
        """Add one event: its TC rows (types [n], hits [n, 14]) against its truth."""
        tc_type = np.asarray(tc_type, dtype=np.int64)
        matched = match_tcs(tc_hits, hit_truth(ev))
        parts = ev.particles
        n_part = len(parts["pt"])
        pt = np.asarray(parts["pt"], dtype=np.float64)
        eta = np.asarray(parts["eta"], dtype=np.float64)
        found = np.zeros(n_part, dtype=bool)
        found_type = np.zeros((4, n_part), dtype=bool)
        good = matched >= 0
        found[matched[good]] = True
        for t in range(4):
            sel = good & (tc_type == t)
            found_type[t, matched[sel]] = True
        ipt = np.digitize(pt, PT_BINS) - 1
        inpt = (ipt >= 0) & (ipt < len(PT_BINS) - 1)
        np.add.at(self.eff_pt_den, ipt[inpt], 1)
        np.add.at(self.eff_pt_num, ipt[inpt & found], 1)
        for t in range(4):
            np.add.at(self.eff_pt_by_type[t], ipt[inpt & found_type[t]], 1)
        ieta = np.digitize(eta, ETA_BINS) - 1
        ineta = (ieta >= 0) & (ieta < len(ETA_BINS) - 1) & (pt > ETA_PT_MIN)
        np.add.at(self.eff_eta_den, ieta[ineta], 1)
        np.add.at(self.eff_eta_num, ieta[ineta & found], 1)
        n_match = np.bincount(matched[good], minlength=n_part) if n_part else np.zeros(0, np.int64)
        dup = good & (n_match[np.where(good, matched, 0)] >= 2) if n_part else np.zeros(len(matched), bool)
        self.n_tc += len(matched)
        self.n_fake += int((~good).sum())
        self.n_dup += int(dup.sum())
        for t in range(4):
            self.n_tc_type[t] += int((tc_type == t).sum())
            self.n_fake_type[t] += int(((tc_type == t) & ~good).sum())
            self.n_dup_type[t] += int(((tc_type == t) & dup).sum())

    def summary(self) -> dict:
        """Rates with their binomial standard errors."""
        def ratio(num, den):
            num = np.asarray(num, dtype=np.float64)
            den = np.asarray(den, dtype=np.float64)
            with np.errstate(invalid="ignore", divide="ignore"):
                r = np.where(den > 0, num / den, np.nan)
                e = np.where(den > 0, np.sqrt(np.clip(r * (1 - r), 0, None) / den), np.nan)
            return r, e
        eff_pt, eff_pt_err = ratio(self.eff_pt_num, self.eff_pt_den)
        eff_eta, eff_eta_err = ratio(self.eff_eta_num, self.eff_eta_den)
        above = PT_BINS[:-1] >= 1.0
        return {
            "pt_bins": PT_BINS.tolist(), "eff_pt": eff_pt.tolist(), "eff_pt_err": eff_pt_err.tolist(),
            "eff_pt_den": self.eff_pt_den.tolist(),
            "eff_pt_by_type": {n: ratio(self.eff_pt_by_type[t], self.eff_pt_den)[0].tolist()
                               for t, n in enumerate(TC_TYPE_NAMES)},
            "eta_bins": ETA_BINS.tolist(), "eff_eta": eff_eta.tolist(), "eff_eta_err": eff_eta_err.tolist(),
            "eff_above_1gev": float(self.eff_pt_num[above].sum() / max(1, self.eff_pt_den[above].sum())),
            "n_tc": self.n_tc,
            "fake_rate": self.n_fake / max(1, self.n_tc),
            "duplicate_rate": self.n_dup / max(1, self.n_tc),
            "by_type": {n: {"n_tc": int(self.n_tc_type[t]),
                            "fake_rate": float(self.n_fake_type[t] / max(1, self.n_tc_type[t])),
                            "duplicate_rate": float(self.n_dup_type[t] / max(1, self.n_tc_type[t]))}
                        for t, n in enumerate(TC_TYPE_NAMES)},
        }
