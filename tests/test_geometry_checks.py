"""Every rejection of lst_load_geometry's table checks, run on the host through lst_check_geometry
(the same checks, no context and no GPU needed): bad module ids, subdetector codes and spacings;
module-map offsets that do not start at 0 or decrease; a module with more than 256 connections;
targets out of range; a pixel map of the wrong bin count, with bad offsets or targets; NULL tables."""
import numpy as np
import pytest

from paper_2207_08207_gb300 import gen, lst


@pytest.fixture(scope="module")
def tables():
    det = gen.make_detector(barrel_only=False, pt_thr=0.8)
    return (det.geom.module_records(), det.conn_off.astype(np.int32), det.conn_tgt.astype(np.int32),
            det.pix_off.astype(np.int32), det.pix_tgt.astype(np.int32))


def _reject(match, *args):
    with pytest.raises(lst.LSTError) as ei:
        lst.check_geometry(*args)
    assert ei.value.code == lst.LST_EINVAL
    assert match in str(ei.value), str(ei.value)


def test_valid_tables_pass(tables):
    mods, co, ct, po, pt = tables
    deg = lst.check_geometry(mods, co, ct, po, pt)
    assert deg == int(np.max(np.diff(co))) and 0 < deg <= 256
    assert lst.check_geometry(mods, co, ct) == deg   # no pixel map


def test_module_table_rejections(tables):
    mods, co, ct, po, pt = tables
    m = mods.copy()
    m["id"][17] = 18
    _reject("ids must equal their index", m, co, ct)
    m = mods.copy()
    m["subdet"][5] = 2
    _reject("bad subdet", m, co, ct)
    m = mods.copy()
    m["spacing"][9] = 0.0
    _reject("spacing must be positive", m, co, ct)
    m = mods.copy()
    m["spacing"][9] = np.nan
    _reject("spacing must be positive", m, co, ct)
    _reject("empty module table", mods[:0], co[:1], ct)


def test_module_map_rejections(tables):
    mods, co, ct, po, pt = tables
    c = co.copy()
    c[0] = 1
    _reject("conn_off[0] != 0", mods, c, ct)
    c = co.copy()
    c[100] = c[101] + 1
    _reject("not monotone", mods, c, ct)
    # one module with 257 connections
    n = mods.size
    c = np.zeros(n + 1, np.int32)
    c[1:] = 257
    t = np.arange(257, dtype=np.int32) % n
    _reject("more than 256 connections", mods, c, t)
    c[1:] = 256
    assert lst.check_geometry(mods, c, t[:256]) == 256
    t = ct.copy()
    t[50] = n
    _reject("conn_tgt out of range", mods, co, t)
    t[50] = -1
    _reject("conn_tgt out of range", mods, co, t)


def test_pixel_map_rejections(tables):
    mods, co, ct, po, pt = tables
    _reject("100 x 128 x 2 bins", mods, co, ct, po[:-1], pt)
    p = po.copy()
    p[0] = 3
    _reject("pix_off[0] != 0", mods, co, ct, p, pt)
    p = po.copy()
    p[1000] = p[1001] + 1
    _reject("pix_off not monotone", mods, co, ct, p, pt)
    t = pt.copy()
    t[7] = mods.size
    _reject("pix_tgt out of range", mods, co, ct, po, t)
