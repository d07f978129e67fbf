"""GB300 engine for HEP-Frame-style event analysis (arXiv:2211.14346): an
ordered cut chain with kinematic reconstruction and detector smearing,
evaluated per event on one GPU behind the C ABI of include/hf.h.

This package is the thin Python side: `_lib` marshals arguments to the C
entry points of the same names, `Engine` wraps a context and converts the
user-level analysis description and numpy / torch columns.  PyTorch is used
only to hold device and pinned host buffers; all computation runs in the
library's CUDA kernels.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib
from ._lib import (HF_FLAG_DEBUG_SYNC, HF_FLAG_NO_SCHED, HF_FLAG_PLAIN, HF_FLAG_PROFILE, HF_FLAG_OVERLAP,  # noqa: F401
                   HF_FLAG_BATCHING, HFError,
                   HF_STATE_DONE, HF_STATE_FAILED, HF_STATE_QUEUED, HF_STATE_RUNNING)

N_RECO = 4
CUDA_STREAM_LEGACY = 1  # cudaStreamLegacy: the handle of the legacy default stream


def _f32(x):
    return float(np.float32(x))


def _cut_struct(cuts):
    arr = (_lib.hf_cut * len(cuts))()
    for i, c in enumerate(cuts):
        name, params = c[0], list(c[1:])
        deps, reorder = 0, 1
        if params and isinstance(params[-1], dict):
            opt = params.pop()
            deps = int(opt.get("dep_mask", 0))
            reorder = int(opt.get("reorderable", 1))
        arr[i].kind = _lib.HF_CUT[name]
        for k, p in enumerate(params[:4]):
            arr[i].params[k] = _f32(p)
        arr[i].dep_mask = deps
        arr[i].reorderable = reorder
    return arr


def columns_struct(ptrs, n_jets_total):
    """hf_columns from raw addresses (host or device)."""
    s = _lib.hf_columns()
    s.jet_off, s.jets, s.btag, s.lep, s.lep_q, s.met = ptrs
    s.n_jets_total = int(n_jets_total)
    return s


class DeviceColumns:
    """A chunk's columns as torch CUDA tensors (device memory only)."""

    def __init__(self, cols, device="cuda"):
        import torch
        self.model = cols.model
        self.n_events = cols.n_events
        self.n_jets_total = cols.n_jets_total
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(device)  # noqa: E731
        self.jet_off = t(cols.jet_off.view(np.int32))
        self.jets = t(cols.jets)
        self.btag = t(cols.btag.view(np.int16))
        self.lep = t(cols.lep)
        self.lep_q = t(cols.lep_q)
        self.met = t(cols.met)
        self._off_host = np.asarray(cols.jet_off, dtype=np.int64)

    def struct(self):
        return columns_struct([x.data_ptr() for x in (self.jet_off, self.jets, self.btag, self.lep,
                                                       self.lep_q, self.met)], self.n_jets_total)

    def nbytes(self):
        return sum(x.numel() * x.element_size() for x in (self.jet_off, self.jets, self.btag, self.lep,
                                                           self.lep_q, self.met))

    def slice(self, lo, hi):
        """Events [lo, hi) as a chunk that shares this chunk's device memory
        (only its rebased jet offsets are a new tensor)."""
        out = DeviceColumns.__new__(DeviceColumns)
        L = 1 if self.model == 1 else 2
        j0, j1 = int(self._off_host[lo]), int(self._off_host[hi])
        out.model = self.model
        out.n_events = hi - lo
        out.n_jets_total = j1 - j0
        out._off_host = self._off_host[lo:hi + 1] - j0
        out.jet_off = (self.jet_off[lo:hi + 1] - j0).contiguous()
        out.jets = self.jets[j0:j1]
        out.btag = self.btag[lo:hi]
        out.lep = self.lep[lo * L:hi * L]
        out.lep_q = self.lep_q[lo * L:hi * L]
        out.met = self.met[lo:hi]
        return out


class PinnedColumns:
    """A chunk's columns in pinned (page-locked) host memory."""

    def __init__(self, cols):
        import torch
        self.model = cols.model
        self.n_events = cols.n_events
        self.n_jets_total = cols.n_jets_total
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()  # noqa: E731
        self.jet_off = t(cols.jet_off.view(np.int32))
        self.jets = t(cols.jets)
        self.btag = t(cols.btag.view(np.int16))
        self.lep = t(cols.lep)
        self.lep_q = t(cols.lep_q)
        self.met = t(cols.met)

    def struct(self):
        return columns_struct([x.data_ptr() for x in (self.jet_off, self.jets, self.btag, self.lep,
                                                       self.lep_q, self.met)], self.n_jets_total)

    def nbytes(self):
        return sum(x.numel() * x.element_size() for x in (self.jet_off, self.jets, self.btag, self.lep,
                                                           self.lep_q, self.met))


class HostColumnsView:
    """hf_columns over numpy arrays (pageable host memory)."""

    def __init__(self, cols):
        self._keep = [np.ascontiguousarray(a) for a in (cols.jet_off, cols.jets, cols.btag, cols.lep,
                                                        cols.lep_q, cols.met)]
        self.n_events = cols.n_events
        self.n_jets_total = cols.n_jets_total

    def struct(self):
        return columns_struct([a.ctypes.data for a in self._keep], self.n_jets_total)


# host layout of hf_record
RECORD_DTYPE = np.dtype([("event", "<u4"), ("level", "<u4"), ("value", "<f4", (4,))])


class DeviceResults:
    """Device result buffers of one run (torch CUDA tensors); record_cap > 0
    adds the per-cut record buffer (24-byte hf_record entries)."""

    def __init__(self, n_events, n_cuts, nbins, device="cuda", record_cap=0):
        import torch
        self.mask = torch.zeros(n_events, dtype=torch.uint8, device=device)
        self.cutflow = torch.zeros(n_cuts + 1, dtype=torch.int64, device=device)
        self.hist = torch.zeros(nbins + 2, dtype=torch.int64, device=device)
        self.n_surv = torch.zeros(n_events, dtype=torch.int16, device=device)
        self.reco = torch.zeros((n_events, N_RECO), dtype=torch.float32, device=device)
        self.recheck_count = torch.zeros(1, dtype=torch.int64, device=device)
        self.record_cap = int(record_cap)
        self.records = torch.zeros((max(1, self.record_cap), 6), dtype=torch.int32, device=device) \
            if self.record_cap else None
        self.n_records = torch.zeros(1, dtype=torch.int64, device=device) if self.record_cap else None
        self.best_v = torch.zeros(n_events, dtype=torch.int16, device=device)

    def struct(self, fields=None):
        s = _lib.hf_results()
        for f in ("mask", "cutflow", "hist", "n_surv", "reco", "recheck_count"):
            if fields is None or f in fields:
                setattr(s, f, getattr(self, f).data_ptr())
        if fields is None or "best_v" in fields:
            s.best_v = self.best_v.data_ptr()
        if self.records is not None and (fields is None or "records" in fields):
            s.records = self.records.data_ptr()
            s.record_cap = self.record_cap
            s.n_records = self.n_records.data_ptr()
        return s

    def numpy(self):
        out = dict(mask=self.mask.cpu().numpy(), cutflow=self.cutflow.cpu().numpy().astype(np.uint64),
                   hist=self.hist.cpu().numpy().astype(np.uint64),
                   n_surv=self.n_surv.cpu().numpy().view(np.uint16), reco=self.reco.cpu().numpy(),
                   recheck_count=int(self.recheck_count.cpu().item()),
                   best_v=self.best_v.cpu().numpy().view(np.uint16))
        if self.records is not None:
            n = int(self.n_records.cpu().item())
            raw = self.records[:min(n, self.record_cap)].cpu().numpy()
            rec = np.ascontiguousarray(raw).view(RECORD_DTYPE).reshape(-1)
            out["n_records"] = n
            out["records"] = rec  # in (event, level) order, as the library writes them
        return out


def analysis_desc(an):
    """hf_analysis_desc of a user-level analysis dict (see synth.analyses);
    returns (desc, cuts): keep cuts alive while desc is in use."""
    cuts = _cut_struct(an["cuts"])
    d = _lib.hf_analysis_desc()
    d.event_model = _lib.HF_MODEL_SEMILEP if an["model"] == "semilep" else _lib.HF_MODEL_DILEP
    d.n_cuts = len(an["cuts"])
    d.cuts = C.cast(cuts, C.POINTER(_lib.hf_cut))
    for k in ("mW", "mt", "sigma_t", "sigma_W", "mH", "sigma_jet", "sigma_met"):
        setattr(d, k, _f32(an[k]))
    d.sigma_lep = _f32(an.get("sigma_lep", 0.0))
    d.per_event = 1 if an.get("per_event", "mean") == "best" else 0
    nb, lo, hi = an["hist"]
    d.hist_nbins, d.hist_lo, d.hist_hi = int(nb), _f32(lo), _f32(hi)
    rec = an.get("record")
    if rec:
        d.record_levels = sum(1 << int(k) for k in rec["levels"])
        vs = list(rec.get("vars", ()))
        if len(vs) > 4:
            raise ValueError("at most 4 recorded variables")
        for i, v in enumerate(vs):
            d.record_vars[i] = _lib.HF_VAR[v]
    return d, cuts


class HLDeviceColumns:
    """Columns of the HL-LHC selection (synth.hl layout) as torch CUDA tensors."""

    def __init__(self, cols, device="cuda"):
        import torch
        self.n_events = cols.n_events
        self.n_jets_total = int(cols.jet_off[-1])
        self.n_leptons_total = int(cols.lep_off[-1])
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(device)  # noqa: E731
        self.jet_off = t(cols.jet_off.view(np.int32))
        self.jets = t(np.asarray(cols.jets, np.float32).reshape(-1, 4))
        self.btag = t(cols.btag.view(np.int16))
        self.lep_off = t(cols.lep_off.view(np.int32))
        self.lep = t(np.asarray(cols.lep, np.float32).reshape(-1, 4))
        self.lep_q = t(cols.lep_q)
        self.lep_flav = t(cols.lep_flav)
        self.met = t(np.asarray(cols.met, np.float32).reshape(-1, 2))

    def struct(self):
        s = _lib.hf_hl_columns()
        (s.jet_off, s.jets, s.btag, s.lep_off, s.lep, s.lep_q, s.lep_flav, s.met) = [
            x.data_ptr() for x in (self.jet_off, self.jets, self.btag, self.lep_off, self.lep, self.lep_q,
                                   self.lep_flav, self.met)]
        s.n_jets_total = self.n_jets_total
        s.n_leptons_total = self.n_leptons_total
        return s

    def nbytes(self):
        return sum(x.numel() * x.element_size() for x in (self.jet_off, self.jets, self.btag, self.lep_off, self.lep,
                                                           self.lep_q, self.lep_flav, self.met))


def hl_desc(met_min=30.0, mll_min=40.0, mtw_min=50.0, dr_iso=0.4, eta_bounds=(2.5, 2.75, 3.5), sigma_met=0.0,
            hist=(50, 0.0, 500.0)):
    """hf_hl_desc of the HL-LHC selection (Sect. 6.1 defaults)."""
    d = _lib.hf_hl_desc()
    d.met_min, d.mll_min, d.mtw_min, d.dr_iso = (_f32(x) for x in (met_min, mll_min, mtw_min, dr_iso))
    for i, b in enumerate(eta_bounds):
        d.eta_bounds[i] = _f32(b)
    d.sigma_met = _f32(sigma_met)
    d.hist_nbins, d.hist_lo, d.hist_hi = int(hist[0]), _f32(hist[1]), _f32(hist[2])
    return d


def fp32_peak(device=0):
    """Measured FP32 throughput of the device (hf_fp32_peak): dict(sm_count,
    tflops_ffma, tflops_ffma2)."""
    lib = _lib.load()
    r = _lib.hf_fp32_peak_result()
    _lib.check(lib.hf_fp32_peak(int(device), C.byref(r)))
    return dict(sm_count=r.sm_count, tflops_ffma=r.tflops_ffma, tflops_ffma2=r.tflops_ffma2)


class Engine:
    """One library context on one GPU."""

    def __init__(self, device=0, flags=0, hbm_budget_bytes=0, max_inflight=0, staging_bytes=0):
        self.lib = _lib.load()
        cfg = _lib.hf_config(device, flags, hbm_budget_bytes, max_inflight, 0, None, staging_bytes)
        ctx = C.c_void_p()
        _lib.check(self.lib.hf_open(C.byref(cfg), C.byref(ctx)))
        self.ctx = ctx
        self._analyses = {}

    def close(self):
        if self.ctx is not None:
            _lib.check(self.lib.hf_close(self.ctx))
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _check(self, st):
        return _lib.check(st, self.ctx)

    def define(self, an) -> int:
        """Registers a user-level analysis (see synth.analyses).  Returns its id."""
        d, cuts = analysis_desc(an)
        aid = C.c_uint32()
        self._check(self.lib.hf_define_cuts(self.ctx, C.byref(d), C.byref(aid)))
        self._analyses[aid.value] = an
        return aid.value

    def results_for(self, aid, n_events, device="cuda", record_cap=None):
        """Result buffers for a run of analysis aid; an analysis that records
        gets room for every possible record (n_events per recorded level)
        unless record_cap says otherwise."""
        an = self._analyses[aid]
        if record_cap is None:
            rec = an.get("record")
            record_cap = n_events * len(set(rec["levels"])) if rec else 0
        return DeviceResults(n_events, len(an["cuts"]), an["hist"][0], device, record_cap)

    def run_device(self, aid, dcols, *, V=1, seed=0, first_event_id=0, out=None, plain=False, stream=None,
                   fields=None):
        """Runs the whole path on device-resident columns; returns DeviceResults."""
        if out is None:
            out = self.results_for(aid, dcols.n_events)
        if stream is None:
            # order the run after torch's uploads and before its reads
            import torch
            stream = torch.cuda.current_stream().cuda_stream or CUDA_STREAM_LEGACY
        cs = dcols.struct()
        rs = out.struct(fields)
        fn = self.lib.hf_run_device_plain if plain else self.lib.hf_run_device
        self._check(fn(self.ctx, aid, C.byref(cs), dcols.n_events, first_event_id, seed, V, C.byref(rs),
                       stream))
        return out

    def run_batch(self, items, *, stream=None):
        """Runs many chunks through one batched launch sequence.

        items: iterable of dicts with keys aid, cols (DeviceColumns), V, seed,
        first_event_id, out (DeviceResults, created when absent).  Returns the
        list of DeviceResults in the order of items."""
        items = list(items)
        arr = (_lib.hf_chunk * max(1, len(items)))()
        outs = []
        for k, it in enumerate(items):
            dc = it["cols"]
            out = it.get("out") or self.results_for(it["aid"], dc.n_events)
            outs.append(out)
            c = arr[k]
            c.analysis_id = it["aid"]
            c.n_variations = it.get("V", 1)
            c.n_events = dc.n_events
            c.first_event_id = it.get("first_event_id", 0)
            c.seed = it.get("seed", 0)
            c.cols = dc.struct()
            c.out = out.struct(it.get("fields"))
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream or CUDA_STREAM_LEGACY
        self._check(self.lib.hf_run_batch(self.ctx, arr, len(items), stream))
        return outs

    def autotune(self, aid, dcols, *, V=1, seed=0):
        """Picks the stage-2 units per tile for this analysis's model and V's
        class from timed runs on dcols (device columns); returns the choice."""
        cs = dcols.struct()
        k = C.c_int32()
        self._check(self.lib.hf_autotune(self.ctx, aid, C.byref(cs), dcols.n_events, V, seed, C.byref(k)))
        return k.value

    def run_hl(self, hcols, desc=None, *, V=1, seed=0, first_event_id=0, channel=True, stream=None, out=None):
        """The HL-LHC multi-region selection on device columns (HLDeviceColumns).
        Returns dict of torch CUDA tensors: counts (6), hist (5, nbins + 2) and,
        with channel=True, channel (N, V) int8."""
        import torch
        d = desc if desc is not None else hl_desc()
        if out is None:
            out = dict(counts=torch.zeros(6, dtype=torch.int64, device="cuda"),
                       hist=torch.zeros((5, d.hist_nbins + 2), dtype=torch.int64, device="cuda"))
            if channel:
                out["channel"] = torch.zeros((hcols.n_events, V), dtype=torch.int8, device="cuda")
        r = _lib.hf_hl_results()
        r.counts = out["counts"].data_ptr()
        r.hist = out["hist"].data_ptr()
        r.channel = out["channel"].data_ptr() if "channel" in out else None
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream or CUDA_STREAM_LEGACY
        cs = hcols.struct()
        self._check(self.lib.hf_run_hl(self.ctx, C.byref(d), C.byref(cs), hcols.n_events, first_event_id, seed, V,
                                       C.byref(r), stream))
        return out

    def device_error(self):
        w = C.c_uint32()
        self._check(self.lib.hf_device_error(self.ctx, C.byref(w)))
        return w.value

    def submit(self, aid, hcols, *, V=1, seed=0, first_event_id=0):
        """Submits host columns (PinnedColumns or HostColumnsView); returns a ticket."""
        cs = hcols.struct()
        t = C.c_uint64()
        self._check(self.lib.hf_submit_chunk(self.ctx, aid, C.byref(cs), hcols.n_events, first_event_id, seed,
                                             V, C.byref(t)))
        return t.value

    def poll(self, ticket):
        s = C.c_int32()
        self._check(self.lib.hf_poll(self.ctx, ticket, C.byref(s)))
        return s.value

    def fetch(self, aid, ticket, n_events, *, fields=("mask", "cutflow", "hist", "n_surv", "reco",
                                                        "recheck_count"), timeout_ms=600000, out=None):
        """Waits for a ticket and copies its results to host numpy arrays."""
        an = self._analyses[aid]
        if out is None:
            out = {}
            if "mask" in fields:
                out["mask"] = np.zeros(n_events, np.uint8)
            if "cutflow" in fields:
                out["cutflow"] = np.zeros(len(an["cuts"]) + 1, np.uint64)
            if "hist" in fields:
                out["hist"] = np.zeros(an["hist"][0] + 2, np.uint64)
            if "n_surv" in fields:
                out["n_surv"] = np.zeros(n_events, np.uint16)
            if "reco" in fields:
                out["reco"] = np.zeros((n_events, N_RECO), np.float32)
            if "recheck_count" in fields:
                out["recheck_count"] = np.zeros(1, np.uint64)
            if "best_v" in fields or an.get("per_event") == "best":
                out["best_v"] = np.zeros(n_events, np.uint16)
        rs = _lib.hf_results()
        for f, a in out.items():
            setattr(rs, f, a.ctypes.data if isinstance(a, np.ndarray) else a.data_ptr())
        self._check(self.lib.hf_fetch_results(self.ctx, ticket, C.byref(rs), timeout_ms))
        return out

    def sched_state(self, aid):
        n = len(self._analyses[aid]["cuts"])
        order = np.zeros(n, np.int32)
        ev, ps, co = (np.zeros(n, np.uint64) for _ in range(3))
        self._check(self.lib.hf_sched_state(self.ctx, aid, order.ctypes.data, ev.ctypes.data, ps.ctypes.data,
                                            co.ctypes.data))
        return dict(order=order, evaluated=ev, passed=ps, cost=co)

    def profile(self, reset=True):
        """Per-phase device times and work counters (context opened with HF_FLAG_PROFILE)."""
        p = _lib.hf_profile_data()
        self._check(self.lib.hf_profile(self.ctx, C.byref(p), 1 if reset else 0))
        return dict(runs=p.runs, ms_stage1=p.ms_stage1, ms_stage2=p.ms_stage2, ms_recheck=p.ms_recheck,
                    launches_stage2=p.launches_stage2, units_stage2=p.units_stage2,
                    events_stage2=p.events_stage2, units_top=list(p.units_top),
                    units_dilep=list(p.units_dilep), pairings_dilep=p.pairings_dilep, cands_top=p.cands_top,
                    batches=p.batches, batched_chunks=p.batched_chunks)

    def set_exec_order(self, aid, order):
        o = np.ascontiguousarray(order, dtype=np.int32)
        self._check(self.lib.hf_set_exec_order(self.ctx, aid, o.ctypes.data))
