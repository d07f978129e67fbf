"""ctypes binding of libhf.so (include/hf.h): the same entry points, argument
marshalling only.  Every step of the path runs in the library's kernels; if
the library cannot be loaded the import fails loudly -- there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhf.so")

HF_OK = 0
HF_EINVAL = -1
HF_ENOMEM = -2
HF_EBUSY = -3
HF_ECUDA = -4
HF_ETIMEOUT = -5
HF_ENOTFOUND = -6
HF_ESTATE = -7
STATUS_NAMES = {0: "HF_OK", -1: "HF_EINVAL", -2: "HF_ENOMEM", -3: "HF_EBUSY", -4: "HF_ECUDA",
                -5: "HF_ETIMEOUT", -6: "HF_ENOTFOUND", -7: "HF_ESTATE"}

HF_FLAG_PLAIN = 1
HF_FLAG_NO_SCHED = 2
HF_FLAG_DEBUG_SYNC = 4
HF_FLAG_PROFILE = 8
HF_FLAG_OVERLAP = 16
HF_FLAG_BATCHING = 32

HF_MODEL_SEMILEP = 1
HF_MODEL_DILEP = 2

HF_CUT = {"njets_min": 1, "nbtag_min": 2, "lep_pt_min": 3, "met_min": 4, "wnu_solvable": 5,
          "hadtop_chi2_max": 6, "lep_os": 7, "dilep_solvable": 8, "higgs_window": 9, "ttbar_chi2_max": 10}

HF_STATE_QUEUED, HF_STATE_RUNNING, HF_STATE_DONE, HF_STATE_FAILED = 0, 1, 2, 3


class hf_config(C.Structure):
    _fields_ = [("device", C.c_int32), ("flags", C.c_uint32), ("hbm_budget_bytes", C.c_uint64),
                ("max_inflight", C.c_uint32), ("reserved", C.c_uint32), ("stream", C.c_void_p),
                ("staging_bytes", C.c_uint64)]


class hf_cut(C.Structure):
    _fields_ = [("kind", C.c_int32), ("params", C.c_float * 4), ("dep_mask", C.c_uint32),
                ("reorderable", C.c_uint8), ("pad", C.c_uint8 * 3)]


# variables of the per-cut recording (HF_VAR_*)
HF_VAR = {"none": 0, "njets": 1, "nbtag": 2, "lep_pt": 3, "met": 4, "reco0": 5, "reco1": 6, "reco2": 7, "reco3": 8}


class hf_analysis_desc(C.Structure):
    _fields_ = [("event_model", C.c_int32), ("n_cuts", C.c_uint32), ("cuts", C.POINTER(hf_cut)),
                ("mW", C.c_float), ("mt", C.c_float), ("sigma_t", C.c_float), ("sigma_W", C.c_float),
                ("mH", C.c_float), ("sigma_jet", C.c_float), ("sigma_met", C.c_float),
                ("hist_nbins", C.c_uint32), ("hist_lo", C.c_float), ("hist_hi", C.c_float),
                ("record_levels", C.c_uint32), ("record_vars", C.c_uint32 * 4), ("sigma_lep", C.c_float),
                ("per_event", C.c_uint32)]


class hf_columns(C.Structure):
    _fields_ = [("jet_off", C.c_void_p), ("jets", C.c_void_p), ("btag", C.c_void_p), ("lep", C.c_void_p),
                ("lep_q", C.c_void_p), ("met", C.c_void_p), ("n_jets_total", C.c_uint64)]


class hf_results(C.Structure):
    _fields_ = [("mask", C.c_void_p), ("cutflow", C.c_void_p), ("hist", C.c_void_p), ("n_surv", C.c_void_p),
                ("reco", C.c_void_p), ("recheck_count", C.c_void_p), ("records", C.c_void_p),
                ("record_cap", C.c_uint64), ("n_records", C.c_void_p), ("best_v", C.c_void_p)]


class hf_chunk(C.Structure):
    _fields_ = [("analysis_id", C.c_uint32), ("n_variations", C.c_uint32), ("n_events", C.c_uint64),
                ("first_event_id", C.c_uint64), ("seed", C.c_uint64), ("cols", hf_columns), ("out", hf_results)]


class hf_hl_columns(C.Structure):
    _fields_ = [("jet_off", C.c_void_p), ("jets", C.c_void_p), ("btag", C.c_void_p), ("lep_off", C.c_void_p),
                ("lep", C.c_void_p), ("lep_q", C.c_void_p), ("lep_flav", C.c_void_p), ("met", C.c_void_p),
                ("n_jets_total", C.c_uint64), ("n_leptons_total", C.c_uint64)]


class hf_hl_desc(C.Structure):
    _fields_ = [("met_min", C.c_float), ("mll_min", C.c_float), ("mtw_min", C.c_float), ("dr_iso", C.c_float),
                ("eta_bounds", C.c_float * 3), ("sigma_met", C.c_float), ("hist_nbins", C.c_uint32),
                ("hist_lo", C.c_float), ("hist_hi", C.c_float)]


class hf_hl_results(C.Structure):
    _fields_ = [("counts", C.c_void_p), ("hist", C.c_void_p), ("channel", C.c_void_p)]


class hf_fp32_peak_result(C.Structure):
    _fields_ = [("sm_count", C.c_int32), ("tflops_ffma", C.c_double), ("tflops_ffma2", C.c_double)]


class hf_profile_data(C.Structure):
    _fields_ = [("runs", C.c_uint64), ("ms_stage1", C.c_double), ("ms_stage2", C.c_double),
                ("ms_recheck", C.c_double), ("launches_stage2", C.c_uint64), ("units_stage2", C.c_uint64),
                ("events_stage2", C.c_uint64), ("units_top", C.c_uint64 * 16), ("units_dilep", C.c_uint64 * 16),
                ("pairings_dilep", C.c_uint64), ("cands_top", C.c_uint64), ("batches", C.c_uint64),
                ("batched_chunks", C.c_uint64)]


_lib = None


def load():
    """Loads libhf.so (built by paper_2211_14346_gb300.build).  Raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("libhf.so not built: run paper_2211_14346_gb300.build.build() "
                          "(nvcc for sm_103a); there is no CPU fallback")
    lib = C.CDLL(LIB_PATH)
    vp, u32, u64, i32 = C.c_void_p, C.c_uint32, C.c_uint64, C.c_int32
    sig = {
        "hf_open": ([C.POINTER(hf_config), C.POINTER(vp)], i32),
        "hf_close": ([vp], i32),
        "hf_last_error": ([vp], C.c_char_p),
        "hf_define_cuts": ([vp, C.POINTER(hf_analysis_desc), C.POINTER(u32)], i32),
        "hf_submit_chunk": ([vp, u32, C.POINTER(hf_columns), u64, u64, u64, u32, C.POINTER(u64)], i32),
        "hf_poll": ([vp, u64, C.POINTER(i32)], i32),
        "hf_fetch_results": ([vp, u64, C.POINTER(hf_results), u32], i32),
        "hf_run_device": ([vp, u32, C.POINTER(hf_columns), u64, u64, u64, u32, C.POINTER(hf_results), vp], i32),
        "hf_run_device_plain": ([vp, u32, C.POINTER(hf_columns), u64, u64, u64, u32, C.POINTER(hf_results), vp],
                                i32),
        "hf_device_error": ([vp, C.POINTER(u32)], i32),
        "hf_sched_state": ([vp, u32, vp, vp, vp, vp], i32),
        "hf_set_exec_order": ([vp, u32, vp], i32),
        "hf_profile": ([vp, C.POINTER(hf_profile_data), i32], i32),
        "hf_run_device_noalloc": ([C.POINTER(hf_analysis_desc), C.POINTER(hf_columns), u64, u64, u64, u32,
                                   C.POINTER(hf_results), vp], i32),
        "hf_run_batch": ([vp, C.POINTER(hf_chunk), u32, vp], i32),
        "hf_autotune": ([vp, u32, C.POINTER(hf_columns), u64, u32, u64, C.POINTER(i32)], i32),
        "hf_fp32_peak": ([i32, C.POINTER(hf_fp32_peak_result)], i32),
        "hf_run_hl": ([vp, C.POINTER(hf_hl_desc), C.POINTER(hf_hl_columns), u64, u64, u64, u32,
                       C.POINTER(hf_hl_results), vp], i32),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def declared_symbols():
    """Names of the entry points this binding marshals (the ones hf.h declares)."""
    return ["hf_open", "hf_close", "hf_last_error", "hf_define_cuts", "hf_submit_chunk", "hf_poll",
            "hf_fetch_results", "hf_run_device", "hf_run_device_plain", "hf_device_error", "hf_sched_state",
            "hf_set_exec_order", "hf_profile", "hf_run_device_noalloc", "hf_run_batch", "hf_autotune",
            "hf_fp32_peak", "hf_run_hl"]


class HFError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


def check(status, ctx=None):
    if status != HF_OK:
        msg = load().hf_last_error(ctx).decode(errors="replace")
        raise HFError(status, msg)
    return status
