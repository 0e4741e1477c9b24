"""Python binding of liblst.so (include/lst.h): argument marshalling only.

Every step of the tracking chain runs in the CUDA library; this module converts numpy arrays or
torch CUDA tensors to the C structs, calls the C ABI, and wraps the library's device outputs as
torch tensors (zero-copy, via ``__cuda_array_interface__``) or copies them to numpy. PyTorch is used
for device memory of caller-side tensors and for streams. There is no CPU fallback: if the library
cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import gen

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblst.so")

LST_OK, LST_EINVAL, LST_ENOMEM, LST_ECUDA, LST_ETIMEOUT, LST_EOVERFLOW_UNRESOLVED, LST_ESTATE = range(7)
LST_MEM_HOST, LST_MEM_DEVICE, LST_MEM_HOST_ASYNC = 0, 1, 2
STAGES = ["md", "ls", "t3", "t5", "pt3", "pt5", "tc", "queue"]
TC_TYPES = ["pT5", "pT3", "T5", "pLS"]

KERNELS = ["bin_sort_gather", "md", "md_compact", "ls", "ls_compact", "t3_pre", "t3_decide", "t3_compact",
           "t5_pre", "t5_decide", "pt3_pre", "pt5_pre", "pt3_decide", "pt5_decide", "t5_clean", "tc_assemble",
           "tc_ext"]

_CONST_FIELDS = ["k", "pt_thr", "sin_max", "z_lum", "d0_max", "n_sigma", "sigma_rphi", "sigma_z", "sigma_r",
                 "chi2_t3", "chi2_t5_c", "chi2_t5_rz", "chi2_pt3_xy", "chi2_pt3_rz", "chi2_pt5_xy",
                 "chi2_pt5_rz", "f_t3", "d0_t3", "c_rel", "c_abs", "dr_min", "pt_cap", "pls_dir_err",
                 "pls_pt_err", "sigma_floor"]


class Config(ctypes.Structure):
    _fields_ = [(f, ctypes.c_float) for f in _CONST_FIELDS] + [
        ("t5_overlap_hits", ctypes.c_int32), ("persistent", ctypes.c_int32), ("use_graph", ctypes.c_int32),
        ("block_ls", ctypes.c_int32), ("warps_px", ctypes.c_int32), ("cap_scale", ctypes.c_float),
        ("max_retries", ctypes.c_int32), ("cycle_budget", ctypes.c_int64), ("half_floats", ctypes.c_int32)]


class EventIn(ctypes.Structure):
    _fields_ = [("x", ctypes.c_void_p), ("y", ctypes.c_void_p), ("z", ctypes.c_void_p),
                ("sensor", ctypes.c_void_p), ("n_hits", ctypes.c_int32), ("pls", ctypes.c_void_p),
                ("n_pls", ctypes.c_int32), ("mem_space", ctypes.c_int32)]


# EventIn as a numpy structured dtype (same offsets and size): a batch of device events is marshalled
# column by column instead of one ctypes structure per event
_EVENT_IN_DTYPE = np.dtype({
    "names": [f for f, _ in EventIn._fields_],
    "formats": ["<u8" if t is ctypes.c_void_p else "<i4" for _, t in EventIn._fields_],
    "offsets": [getattr(EventIn, f).offset for f, _ in EventIn._fields_],
    "itemsize": ctypes.sizeof(EventIn)})


def _tensor_events_in(events, host_async):
    """The EventIn records of a batch of events given as dicts of torch tensors, as a numpy array.
    CUDA tensors are device inputs; CPU tensors (pinned or pageable) are host inputs, held until
    sync with host_async, else copied before the call returns."""
    buf = np.zeros(len(events), dtype=_EVENT_IN_DTYPE)
    for f in ("x", "y", "z", "sensor"):
        buf[f] = [ev[f].data_ptr() for ev in events]
    buf["n_hits"] = [ev["x"].shape[0] for ev in events]
    n_pls = [int(ev.get("n_pls", 0)) for ev in events]
    buf["n_pls"] = n_pls
    buf["pls"] = [ev["pls"].data_ptr() if k else 0 for ev, k in zip(events, n_pls)]
    host = LST_MEM_HOST_ASYNC if host_async else LST_MEM_HOST
    buf["mem_space"] = [LST_MEM_DEVICE if ev["x"].is_cuda else host for ev in events]
    return buf


def _addr(a):
    """Address of a contiguous numpy array's data (the buffer protocol where the array is writable:
    cheaper than the .ctypes attribute, which stays the fallback)."""
    try:
        return ctypes.addressof(ctypes.c_char.from_buffer(a))
    except (TypeError, ValueError, BufferError):
        return a.ctypes.data


def _host_events_in(events, host_async):
    """The EventIn records of a batch of host events (gen.Event objects with numpy arrays), as a
    numpy array, and the contiguous arrays they point to (to be kept alive until sync)."""
    buf = np.zeros(len(events), dtype=_EVENT_IN_DTYPE)
    keep = []
    cols = {f: [] for f in ("x", "y", "z", "sensor", "pls", "n_hits", "n_pls")}
    asc, f32, i32 = np.ascontiguousarray, np.float32, np.int32
    for ev in events:
        x, y, z = asc(ev.x, dtype=f32), asc(ev.y, dtype=f32), asc(ev.z, dtype=f32)
        s = asc(ev.sensor, dtype=i32)
        k = ev.n_pls
        p = asc(ev.pls) if k else None
        keep += (x, y, z, s, p)
        cols["x"].append(_addr(x)); cols["y"].append(_addr(y)); cols["z"].append(_addr(z))
        cols["sensor"].append(_addr(s)); cols["pls"].append(_addr(p) if k else 0)
        cols["n_hits"].append(x.shape[0]); cols["n_pls"].append(k)
    for f, v in cols.items():
        buf[f] = v
    buf["mem_space"] = LST_MEM_HOST_ASYNC if host_async else LST_MEM_HOST
    return buf, keep


class Counts(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in ("n_hits", "n_pls", "n_md", "n_ls", "n_t3", "n_t5", "n_pt3",
                                              "n_pt5", "n_tc")] + [
        ("n_tc_type", ctypes.c_int32 * 4), ("overflow", ctypes.c_int32 * 8), ("recheck", ctypes.c_int32 * 8),
        ("retries", ctypes.c_int32), ("status", ctypes.c_int32), ("n_tc_ext", ctypes.c_int32),
        ("n_ls_pairs", ctypes.c_int64)]

    def as_dict(self):
        d = {n: getattr(self, n) for n in ("n_hits", "n_pls", "n_md", "n_ls", "n_t3", "n_t5", "n_pt3", "n_pt5",
                                           "n_tc", "retries", "status", "n_tc_ext", "n_ls_pairs")}
        d["n_tc_type"] = dict(zip(TC_TYPES, list(self.n_tc_type)))
        d["overflow"] = dict(zip(STAGES, list(self.overflow)))
        d["recheck"] = dict(zip(STAGES, list(self.recheck)))
        return d


# (field, dtype code, length key) of lst_event_out after `counts`
OUT_FIELDS = [
    ("md_hit_lo", "i4", "n_md"), ("md_hit_up", "i4", "n_md"), ("md_module", "i4", "n_md"),
    ("md_dphichange", "f4", "n_md"), ("md_pt_est", "f4", "n_md"),
    ("ls_md_in", "i4", "n_ls"), ("ls_md_out", "i4", "n_ls"), ("ls_z0", "f4", "n_ls"), ("ls_dphi", "f4", "n_ls"),
    ("t3_ls_in", "i4", "n_t3"), ("t3_ls_out", "i4", "n_t3"), ("t3_r", "f4", "n_t3"), ("t3_xc", "f4", "n_t3"),
    ("t3_yc", "f4", "n_t3"), ("t3_chi2_rz", "f4", "n_t3"), ("t3_pt_est", "f4", "n_t3"),
    ("t5_t3_in", "i4", "n_t5"), ("t5_t3_out", "i4", "n_t5"), ("t5_kappa_in", "f4", "n_t5"),
    ("t5_kappa_out", "f4", "n_t5"), ("t5_kappa_fit", "f4", "n_t5"), ("t5_chi2_c", "f4", "n_t5"),
    ("t5_chi2_rz", "f4", "n_t5"), ("t5_eta", "f4", "n_t5"), ("t5_phi", "f4", "n_t5"), ("t5_pt", "f4", "n_t5"),
    ("pt3_pls", "i4", "n_pt3"), ("pt3_t3", "i4", "n_pt3"), ("pt3_chi2_xy", "f4", "n_pt3"),
    ("pt3_chi2_rz", "f4", "n_pt3"),
    ("pt5_pls", "i4", "n_pt5"), ("pt5_t5", "i4", "n_pt5"), ("pt5_chi2_xy", "f4", "n_pt5"),
    ("pt5_chi2_rz", "f4", "n_pt5"),
    ("tc_type", "i4", "n_tc"), ("tc_obj", "i4", "n_tc"), ("tc_hits", "i4", "n_tc14"),
    ("tc_pt", "f4", "n_tc"), ("tc_eta", "f4", "n_tc"), ("tc_phi", "f4", "n_tc"),
    ("tc_ext_t3", "i4", "n_tc"), ("tc_ext_n_md", "i4", "n_tc"), ("tc_ext_hits", "i4", "n_tc4"),
    ("tc_ext_chi2_c", "f4", "n_tc"), ("tc_ext_chi2_rz", "f4", "n_tc"),
    # binary16 twins of the output-only columns (lst_config.half_floats = 1; NULL otherwise)
    ("md_dphichange_h", "f2", "n_md"), ("md_pt_est_h", "f2", "n_md"), ("ls_z0_h", "f2", "n_ls"),
    ("ls_dphi_h", "f2", "n_ls"), ("t3_xc_h", "f2", "n_t3"), ("t3_yc_h", "f2", "n_t3"),
    ("t3_chi2_rz_h", "f2", "n_t3"), ("t3_pt_est_h", "f2", "n_t3"), ("t5_kappa_in_h", "f2", "n_t5"),
    ("t5_kappa_out_h", "f2", "n_t5"), ("t5_chi2_rz_h", "f2", "n_t5"), ("pt3_chi2_xy_h", "f2", "n_pt3"),
    ("pt3_chi2_rz_h", "f2", "n_pt3"), ("pt5_chi2_xy_h", "f2", "n_pt5"), ("pt5_chi2_rz_h", "f2", "n_pt5"),
]
HALF_FIELDS = [f for f, t, _ in OUT_FIELDS if t == "f2"]


class EventOut(ctypes.Structure):
    _fields_ = [("counts", Counts)] + [(f, ctypes.c_void_p) for f, _, _ in OUT_FIELDS]


_lib = None
_lib_lock = threading.Lock()


def lib():
    """Load liblst.so (building it first if the sources are newer). Raises if it cannot be loaded."""
    global _lib
    with _lib_lock:
        if _lib is not None:
            return _lib
        from . import _build
        if not _build.up_to_date():
            _build.build()
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("liblst.so is missing: run paper_2207_08207_gb300._build.build()")
        L = ctypes.CDLL(LIB_PATH)
        L.lst_config_default.argtypes = [ctypes.POINTER(Config)]
        L.lst_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(Config), ctypes.c_int]
        L.lst_destroy.argtypes = [ctypes.c_void_p]
        L.lst_load_geometry.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32]
        L.lst_reserve.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]
        L.lst_run_events.argtypes = [ctypes.c_void_p, ctypes.POINTER(EventIn), ctypes.c_int32,
                                     ctypes.POINTER(EventOut), ctypes.c_void_p]
        L.lst_sync.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
        L.lst_query.argtypes = [ctypes.c_void_p]
        L.lst_bin_hits.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                   ctypes.c_void_p, ctypes.c_void_p]
        L.lst_bin_hits_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                           ctypes.c_void_p, ctypes.c_void_p]
        L.lst_get_counts.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(Counts)]
        L.lst_copy_tc.argtypes = [ctypes.c_void_p, ctypes.c_int32] + [ctypes.c_void_p] * 6
        L.lst_copy_tc_ext.argtypes = [ctypes.c_void_p, ctypes.c_int32] + [ctypes.c_void_p] * 5
        L.lst_set_timing.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.lst_get_stage_ms.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
        L.lst_tc_total.argtypes = [ctypes.c_void_p]
        L.lst_tc_total.restype = ctypes.c_int64
        L.lst_copy_tc_all.argtypes = [ctypes.c_void_p] + [ctypes.c_void_p] * 7
        L.lst_predict_bytes.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_int64]
        L.lst_predict_bytes.restype = ctypes.c_int64
        L.lst_get_kernel_ms.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32]
        L.lst_launch_count.argtypes = [ctypes.c_void_p]
        L.lst_launch_count.restype = ctypes.c_int64
        L.lst_last_error.argtypes = [ctypes.c_void_p]
        L.lst_last_error.restype = ctypes.c_char_p
        L.lst_selftest_bounded_wait.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int32)]
        L.lst_check_geometry.argtypes = [ctypes.c_void_p, ctypes.c_int32] + [ctypes.c_void_p] * 4 + \
            [ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]
        _lib = L
        return L


def default_config(**overrides) -> Config:
    c = Config()
    lib().lst_config_default(ctypes.byref(c))
    for k, v in overrides.items():
        setattr(c, k, v)
    return c


class LSTError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"LST error {code}: {msg}")
        self.code = code


def _ptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return ctypes.c_void_p(a.data_ptr())
    return ctypes.c_void_p(a.ctypes.data)


class _CudaArray:
    def __init__(self, ptr, n, typestr):
        self.__cuda_array_interface__ = {"shape": (int(n),), "typestr": "<" + typestr,
                                         "data": (int(ptr or 0), False), "version": 3, "strides": None}


class Context:
    """One library context: resident geometry of a detector, arenas, one stream."""

    def __init__(self, det: gen.Detector, config: Config | None = None, device: int = 0, **overrides):
        self._L = lib()
        if config is None:
            config = default_config(pt_thr=float(np.float32(det.pt_thr)), **overrides)
        self.config = config
        h = ctypes.c_void_p()
        rc = self._L.lst_create(ctypes.byref(h), ctypes.byref(config), device)
        if rc != LST_OK:
            raise LSTError(rc, self._L.lst_last_error(None).decode())
        self._h = h
        self.det = det
        self.device = device
        mods = np.ascontiguousarray(det.geom.module_records())
        co = np.ascontiguousarray(det.conn_off, dtype=np.int32)
        ct = np.ascontiguousarray(det.conn_tgt, dtype=np.int32)
        po = np.ascontiguousarray(det.pix_off, dtype=np.int32)
        pt = np.ascontiguousarray(det.pix_tgt, dtype=np.int32)
        n_pix = int(po.size - 1) if pt.size else 0
        self._check(self._L.lst_load_geometry(self._h, _ptr(mods), det.n_mods, _ptr(co), _ptr(ct),
                                              _ptr(po) if n_pix else None, _ptr(pt) if pt.size else None, n_pix))
        self._keep = []
        self._outs = None
        self._n_ev = 0

    def close(self):
        if getattr(self, "_h", None):
            self._L.lst_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != LST_OK:
            raise LSTError(rc, self._L.lst_last_error(self._h).decode())
        return rc

    def reserve(self, n_events, max_hits, max_pls):
        self._check(self._L.lst_reserve(self._h, n_events, max_hits, max_pls))

    # -- running ----------------------------------------------------------------------------
    def submit(self, events, stream=None, host_async=False):
        """Enqueue a batch. `events`: gen.Event objects (host numpy) or dicts of torch tensors with
        keys x, y, z, sensor, pls (uint8/int32 tensor viewing lst_pls records or None) and n_pls;
        CUDA tensors are device inputs, CPU tensors host inputs.
        host_async: pass host events as LST_MEM_HOST_ASYNC (the arrays are held until sync; pinned
        arrays are then read by the device in place instead of being packed on the host)."""
        n = len(events)
        is_dict = [isinstance(ev, dict) for ev in events]
        if n and all(is_dict):            # dicts of tensors: the records built one column at a time
            buf = _tensor_events_in(events, host_async)
            arr = ctypes.cast(buf.ctypes.data, ctypes.POINTER(EventIn))
            keep = [buf, list(events)]
        elif n and not any(is_dict):      # host events
            buf, keep = _host_events_in(events, host_async)
            arr = ctypes.cast(buf.ctypes.data, ctypes.POINTER(EventIn))
            keep.append(buf)
        else:                             # a mixed batch: record by record
            arr, keep = self._events_in(events, host_async)
        outs = (EventOut * n)()
        st = None
        if stream is not None:
            st = ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
        self._check(self._L.lst_run_events(self._h, arr, n, outs, st))
        self._keep = keep
        self._outs = outs
        self._n_ev = n
        return outs

    @staticmethod
    def _events_in(events, host_async):
        """EventIn records of a mixed batch (dicts of tensors and gen.Event objects), one by one."""
        n = len(events)
        arr = (EventIn * n)()
        keep = []
        for i, ev in enumerate(events):
            if isinstance(ev, dict):
                x, y, z, s, p = ev["x"], ev["y"], ev["z"], ev["sensor"], ev.get("pls")
                n_pls = int(ev.get("n_pls", 0))
                mem = LST_MEM_DEVICE if x.is_cuda else (LST_MEM_HOST_ASYNC if host_async else LST_MEM_HOST)
            else:
                x = np.ascontiguousarray(ev.x, dtype=np.float32)
                y = np.ascontiguousarray(ev.y, dtype=np.float32)
                z = np.ascontiguousarray(ev.z, dtype=np.float32)
                s = np.ascontiguousarray(ev.sensor, dtype=np.int32)
                p = np.ascontiguousarray(ev.pls) if ev.n_pls else None
                n_pls = ev.n_pls
                mem = LST_MEM_HOST_ASYNC if host_async else LST_MEM_HOST
            keep += [x, y, z, s, p]
            nh = int(x.shape[0]) if hasattr(x, "shape") else len(x)
            arr[i] = EventIn(_ptr(x), _ptr(y), _ptr(z), _ptr(s), nh, _ptr(p) if n_pls else None, n_pls, mem)
        return arr, keep

    def sync(self):
        status = np.zeros(max(self._n_ev, 1), dtype=np.int32)
        rc = self._L.lst_sync(self._h, _ptr(status))
        self._keep = []
        if rc != LST_OK:
            raise LSTError(rc, self._L.lst_last_error(self._h).decode())
        return status[: self._n_ev]

    def query(self) -> bool:
        rc = self._L.lst_query(self._h)
        if rc < 0:
            raise LSTError(-rc, self._L.lst_last_error(self._h).decode())
        return rc == 1

    def run(self, events, stream=None):
        self.submit(events, stream)
        self.sync()
        return self

    # -- results ----------------------------------------------------------------------------
    def counts(self, ev: int = 0) -> dict:
        c = Counts()
        self._check(self._L.lst_get_counts(self._h, ev, ctypes.byref(c)))
        return c.as_dict()

    def device_arrays(self, ev: int = 0) -> dict:
        """Zero-copy torch views of event `ev`'s device outputs (valid until the next run)."""
        import torch
        o = self._outs[ev]
        c = o.counts
        lens = {k: getattr(c, k) for k in ("n_md", "n_ls", "n_t3", "n_t5", "n_pt3", "n_pt5", "n_tc")}
        lens["n_tc14"] = c.n_tc * 14
        lens["n_tc4"] = c.n_tc * 4
        out = {}
        for f, t, nk in OUT_FIELDS:
            n = lens[nk]
            ptr = getattr(o, f)
            if n == 0 or not ptr:
                dt = {"i4": torch.int32, "f4": torch.float32, "f2": torch.float16}[t]
                out[f] = torch.zeros(0, dtype=dt, device=f"cuda:{self.device}")
            else:
                out[f] = torch.as_tensor(_CudaArray(ptr, n, t), device=f"cuda:{self.device}")
        out["tc_hits"] = out["tc_hits"].view(-1, 14)
        out["tc_ext_hits"] = out["tc_ext_hits"].view(-1, 4)
        return out

    def results(self, ev: int = 0) -> dict:
        """Host (numpy) copies of event `ev`'s objects."""
        d = {k: v.cpu().numpy() for k, v in self.device_arrays(ev).items()}
        d["counts"] = self.counts(ev)
        return d

    def copy_tc(self, ev: int = 0) -> dict:
        n = self.counts(ev)["n_tc"]
        out = {"type": np.zeros(n, np.int32), "obj": np.zeros(n, np.int32), "hits": np.zeros((n, 14), np.int32),
               "pt": np.zeros(n, np.float32), "eta": np.zeros(n, np.float32), "phi": np.zeros(n, np.float32)}
        self._check(self._L.lst_copy_tc(self._h, ev, _ptr(out["type"]), _ptr(out["obj"]), _ptr(out["hits"]),
                                        _ptr(out["pt"]), _ptr(out["eta"]), _ptr(out["phi"])))
        return out

    def copy_tc_ext(self, ev: int = 0) -> dict:
        """Event `ev`'s track extensions (one per TC row) in host memory."""
        n = self.counts(ev)["n_tc"]
        out = {"t3": np.zeros(n, np.int32), "n_md": np.zeros(n, np.int32), "hits": np.zeros((n, 4), np.int32),
               "chi2_c": np.zeros(n, np.float32), "chi2_rz": np.zeros(n, np.float32)}
        self._check(self._L.lst_copy_tc_ext(self._h, ev, _ptr(out["t3"]), _ptr(out["n_md"]), _ptr(out["hits"]),
                                            _ptr(out["chi2_c"]), _ptr(out["chi2_rz"])))
        return out

    def copy_tc_all(self, out=None) -> dict:
        """Every track candidate of the last run, one transfer per array. `out`: optional dict of
        preallocated (e.g. pinned) numpy arrays large enough for the batch."""
        n = int(self._L.lst_tc_total(self._h))
        if out is None:
            out = {"offsets": np.zeros(self._n_ev + 1, np.int32), "type": np.zeros(n, np.int32),
                   "obj": np.zeros(n, np.int32), "hits": np.zeros((n, 14), np.int32), "pt": np.zeros(n, np.float32),
                   "eta": np.zeros(n, np.float32), "phi": np.zeros(n, np.float32)}
        self._check(self._L.lst_copy_tc_all(self._h, _ptr(out["offsets"]), _ptr(out["type"]), _ptr(out["obj"]),
                                            _ptr(out["hits"]), _ptr(out["pt"]), _ptr(out["eta"]), _ptr(out["phi"])))
        out["n"] = n
        return out

    def set_timing(self, on=True):
        self._check(self._L.lst_set_timing(self._h, 1 if on else 0))

    def stage_ms(self) -> dict:
        a = np.zeros(9, dtype=np.float32)
        self._check(self._L.lst_get_stage_ms(self._h, _ptr(a)))
        return dict(zip(STAGES + ["total"], a.tolist()))

    def bin_hits(self, sensor_dev, order_dev, offsets_dev, stream=None):
        """Standalone hit binning of one event (torch CUDA int32 tensors)."""
        _check_dev_i32("sensor", sensor_dev, 0)
        _check_dev_i32("order", order_dev, int(sensor_dev.numel()))
        _check_dev_i32("offsets", offsets_dev, 2 * self.det.n_mods + 1)
        st = None
        if stream is not None:
            st = ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
        self._check(self._L.lst_bin_hits(self._h, _ptr(sensor_dev), int(sensor_dev.numel()), _ptr(order_dev),
                                         _ptr(offsets_dev), st))

    def launch_count(self) -> int:
        return int(self._L.lst_launch_count(self._h))

    def predict_bytes(self, n_events, n_hits, n_pls) -> int:
        v = int(self._L.lst_predict_bytes(self._h, int(n_events), int(n_hits), int(n_pls)))
        if v < 0:
            raise LSTError(-v, "lst_predict_bytes")
        return v

    def kernel_ms(self) -> dict:
        a = np.zeros(len(KERNELS), dtype=np.float32)
        self._L.lst_get_kernel_ms(self._h, _ptr(a), len(KERNELS))
        return dict(zip(KERNELS, a.tolist()))

    def kernel_algorithmic_bytes(self, kernel, counts, n_hits, n_pls) -> int:
        return algorithmic_bytes(kernel, counts, n_hits, n_pls, self.det.n_mods)


def _check_dev_i32(name, t, n_min):
    """The C call writes and reads through raw pointers: each tensor must be a contiguous CUDA int32
    tensor holding at least n_min elements."""
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.int32 and t.is_contiguous()):
        raise LSTError(LST_EINVAL, f"{name}: expected a contiguous CUDA int32 tensor")
    if t.numel() < n_min:
        raise LSTError(LST_EINVAL, f"{name}: {t.numel()} elements, at least {n_min} needed")


def bin_hits_noalloc(sensor_dev, n_sensors, order_dev, offsets_dev, stream=None):
    """Hit binning without any device allocation (lst_bin_hits_noalloc): for callers whose device
    memory is fixed up front. torch CUDA int32 tensors; at most 65536 sensors."""
    n_hits = int(sensor_dev.numel()) if hasattr(sensor_dev, "numel") else -1
    _check_dev_i32("sensor", sensor_dev, 0)
    _check_dev_i32("order", order_dev, n_hits)
    _check_dev_i32("offsets", offsets_dev, int(n_sensors) + 1)
    L = lib()
    st = None
    if stream is not None:
        st = ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    rc = L.lst_bin_hits_noalloc(_ptr(sensor_dev), int(sensor_dev.numel()), int(n_sensors), _ptr(order_dev),
                                _ptr(offsets_dev), st)
    if rc != LST_OK:
        raise LSTError(rc, L.lst_last_error(None).decode())


def check_geometry(mods, conn_off, conn_tgt, pix_off=None, pix_tgt=None):
    """lst_check_geometry on host tables (needs no GPU): returns the largest module-map degree or
    raises LSTError(LST_EINVAL) with the library's reason."""
    L = lib()
    mods = np.ascontiguousarray(mods)
    co = np.ascontiguousarray(conn_off, dtype=np.int32)
    ct = np.ascontiguousarray(conn_tgt, dtype=np.int32)
    n_pix = 0
    po = pt = None
    if pix_off is not None:
        po = np.ascontiguousarray(pix_off, dtype=np.int32)
        pt = np.ascontiguousarray(pix_tgt, dtype=np.int32)
        n_pix = int(po.size - 1)
    deg = ctypes.c_int32(-1)
    rc = L.lst_check_geometry(_ptr(mods) if mods.size else None, int(mods.size), _ptr(co) if co.size else None,
                              _ptr(ct) if ct.size else None, _ptr(po) if po is not None else None,
                              _ptr(pt) if pt is not None and pt.size else None, n_pix, ctypes.byref(deg))
    if rc != LST_OK:
        raise LSTError(rc, L.lst_last_error(None).decode())
    return int(deg.value)


def selftest_bounded_wait(device: int = 0) -> int:
    """Number of block waits that gave up in the library's bounded-wait self-test (>= 1 when the
    bound works); raises on a CUDA error."""
    n = ctypes.c_int32(0)
    rc = lib().lst_selftest_bounded_wait(device, ctypes.byref(n))
    if rc != LST_OK:
        raise LSTError(rc, "lst_selftest_bounded_wait failed")
    return int(n.value)


def exported_symbols():
    """Names of every function include/lst.h declares."""
    import re
    hdr = os.path.join(os.path.dirname(_HERE), "include", "lst.h")
    with open(hdr) as f:
        txt = f.read()
    return sorted(set(re.findall(r"^\s*(?:int|void|int64_t|const char\*)\s+(lst_[a-z_]+)\s*\(", txt, re.M)))


def algorithmic_bytes(kernel, counts, n_hits, n_pls, n_mods) -> int:
    """Compulsory HBM bytes of one launch of a timed kernel: every input element it needs read once,
    every output it produces written once (sizes of the SoA fields). `counts` is the list of
    per-event count dicts of the launch's batch; n_mods the detector's module count."""
    s = lambda k: sum(c[k] for c in counts)
    n_md, n_ls, n_t3, n_t5 = s("n_md"), s("n_ls"), s("n_t3"), s("n_t5")
    n_pt3, n_pt5, n_tc = s("n_pt3"), s("n_pt5"), s("n_tc")
    n_mod = n_mods * len(counts)
    table = {
        # binned x, y, z (12 B) + input index (4 B) written, sensor offsets read
        "bin_sort_gather": n_hits * (16 + 12 + 4) + 2 * n_mod * 4,
        # hit coordinates read once, MD slots written (lo, up, dphichange, pt_est)
        "md": n_hits * 12 + 2 * n_mod * 4 + n_md * 16,
        "md_compact": n_md * (16 + 41) + n_hits * 16,
        # MD anchors (x, y, z, r, s_thr, endcap: 21 B) read once, LS slots written (16 B)
        "ls": n_md * 21 + n_mod * 12 + n_ls * 16,
        "ls_compact": n_ls * (16 + 16 + 24),
        # LS (8 B) + MD anchors read, queue pairs written (8 B per surviving candidate)
        "t3_pre": n_ls * 8 + n_md * 21 + n_t3 * 8,
        "t3_decide": n_t3 * (8 + 3 * 12 + 28),
        "t3_compact": n_t3 * (28 + 40),
        "t5_pre": n_t3 * 8 + n_t5 * 8,
        "t5_decide": n_t5 * (8 + 5 * 13 + 40),
        # seeds (48 B) + T3 member MDs (12 B) + anchors, passing pairs written
        "pt3_pre": n_pls * 48 + n_t3 * 12 + n_md * 17 + n_pt3 * 8,
        "pt5_pre": n_pls * 48 + n_t5 * 20 + n_md * 17 + n_pt5 * 8,
        "pt3_decide": n_pt3 * (8 + 48 + 3 * 13 + 20),
        "pt5_decide": n_pt5 * (8 + 48 + 5 * 13 + 20),
        "t5_clean": n_t5 * (20 + 32 + 4) + n_hits * 8,
        "tc_assemble": n_tc * (4 + 4 + 56 + 12) + n_pls * 12 + n_t5 * 12,
    }
    return int(table.get(kernel, 0))
