/*
 * hf.h -- C ABI of the GB300 event-analysis engine: an ordered cut chain
 * with kinematic reconstruction and detector smearing, evaluated per event
 * over millions of independent collision events on one GPU.
 *
 * Method: HEP-Frame (A. Pereira, A. Onofre, A. Proenca, arXiv:2211.14346).
 *   - A user analysis is an ordered list of cuts ("propositions"); each event
 *     is tested against them in order and stops at the first failing one; an
 *     event passing all cuts is selected (Sect. 3, registration of cuts with
 *     the analysis in user order; Sect. 6.1, cut example).
 *   - Semileptonic reconstruction: neutrino p_z from the W-mass constraint
 *     with the missing transverse momentum (MET) as the neutrino pT, and the
 *     jet-triplet chi-square of Eq. 1 (Sect. 6.2), hadronic-top term.
 *   - Dilepton ttH reconstruction: two neutrinos from the W-mass (80.4 GeV)
 *     and top-mass (172.5 GeV) constraints with MET split between them, over
 *     all b-jet/lepton pairings, the best solution kept; no solution rejects
 *     the event; the Higgs candidate from the two remaining b-jets closest to
 *     125 GeV (Sect. 4).
 *   - N detector-resolution pseudo-experiments ("variations") per event
 *     (Sect. 4), drawn from Philox4x32-10 keyed by (seed, event, variation).
 *   - Per-cut counts (cut flow) and user histograms (Appendix).
 *
 * Terminology: a "unit" is one (event, variation) pair; V variations per
 * event (V = 1 and zero widths = unsmeared).  The cut flow counts units.
 *
 * Conventions for every entry point:
 *   - Return value: HF_OK (0) or a negative hf_status.  No entry point aborts,
 *     throws or exits; hf_last_error() gives a message for the calling thread.
 *   - Pointers documented as "host" are CPU memory, "device" are CUDA device
 *     memory on the context's GPU.  The library never frees caller memory.
 *   - All entry points are thread-safe (one internal mutex per context).
 */
#ifndef HF_H
#define HF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t hf_status;
#define HF_OK 0
#define HF_EINVAL (-1)    /* invalid argument, descriptor or event columns   */
#define HF_ENOMEM (-2)    /* device or pinned host allocation failed          */
#define HF_EBUSY (-3)     /* admission refused: HBM budget or slots full; retry */
#define HF_ECUDA (-4)     /* a CUDA call failed; see hf_last_error            */
#define HF_ETIMEOUT (-5)  /* a bounded wait expired                            */
#define HF_ENOTFOUND (-6) /* unknown ticket or analysis id                     */
#define HF_ESTATE (-7)    /* call not valid in the current state               */

typedef struct hf_ctx hf_ctx;

/* Largest number of smearing variations per event of any entry point (the
 * units of one event share one stage-2 tile in shared memory). */
#define HF_MAX_VARIATIONS 4096u

/* hf_config.flags */
#define HF_FLAG_PLAIN 1u      /* run every chunk with the plain one-thread-per-event kernel */
#define HF_FLAG_NO_SCHED 2u   /* keep the user order for execution (no reordering)         */
#define HF_FLAG_DEBUG_SYNC 4u /* synchronise after every launch and check errors           */
#define HF_FLAG_OVERLAP 16u   /* run the per-multiplicity stage-2 kernels of a run on side
                                 streams so that they overlap (default: one after another)  */
#define HF_FLAG_BATCHING 32u  /* continuous batching of hf_submit_chunk: a dispatcher thread
                                 of the context launches all queued chunks as one batch
                                 (hf_run_batch's kernels) whenever fewer than two batches are
                                 unfinished; chunks arriving meanwhile join the next batch */

typedef struct {
    int32_t device;            /* CUDA device ordinal                                   */
    uint32_t flags;            /* HF_FLAG_*                                             */
    uint64_t hbm_budget_bytes; /* admission budget for in-flight chunks (0 = 80% of free) */
    uint32_t max_inflight;     /* maximum in-flight tickets (0 = 64)                    */
    uint32_t reserved;
    void* stream;              /* optional cudaStream_t to order work after (NULL = own) */
    uint64_t staging_bytes;    /* pinned staging ring for columns in pageable host memory
                                  (0 = none; the input side of the overlap of reading and
                                  processing that Sect. 5.1 gets from reader threads):
                                  hf_submit_chunk copies such a column into the
                                  ring on the host and from there asynchronously, so that the
                                  caller may reuse that buffer when the call returns; columns
                                  in pinned memory, or larger than the ring, are copied
                                  straight from the caller's buffer (which must then stay
                                  valid until the ticket is done).  Ring space is reused once
                                  the copy that filled it has completed (the host waits for
                                  it when the ring is full).                                */
} hf_config;

/* Opens a context on cfg->device: the state an analysis run needs on one
 * GPU -- registered analyses, their cut schedulers, scratch memory, streams
 * and in-flight chunks (the role of HEP-Frame's generated analysis skeleton
 * and its run-time thread pool, Sect. 2 and Sect. 5.1, here for one device).
 * cfg may be NULL (device 0, defaults).  *out receives the context; release
 * it with hf_close.  Errors: HF_EINVAL (bad device), HF_ECUDA, HF_ENOMEM. */
hf_status hf_open(const hf_config* cfg, hf_ctx** out);

/* Closes the context: waits (bounded, 60 s) for in-flight work, frees all
 * device and pinned memory it owns.  ctx may be NULL.  Returns HF_ETIMEOUT if
 * work did not finish in time (memory is then leaked, not freed under a
 * running kernel). */
hf_status hf_close(hf_ctx* ctx);

/* Message of the last error on the calling thread (static storage, never NULL). */
const char* hf_last_error(hf_ctx* ctx);

/* ------------------------------------------------------------------ */
/* Analysis description (hf_define_cuts).                               */
/* ------------------------------------------------------------------ */
#define HF_MODEL_SEMILEP 1 /* one lepton; needs HF_CUT_W_NU_SOLVABLE and HF_CUT_HADTOP_CHI2_MAX
                              or HF_CUT_TTBAR_CHI2_MAX */
#define HF_MODEL_DILEP 2   /* two leptons; needs HF_CUT_DILEP_SOLVABLE and HF_CUT_HIGGS_WINDOW   */

/* Cut kinds.  Each is a pure predicate of one unit, so any user order gives
 * the same selected units (only the cut flow, reported in user order, changes). */
#define HF_CUT_NJETS_MIN 1       /* n_jets >= params[0]                                    */
#define HF_CUT_NBTAG_MIN 2       /* b-tagged jets >= params[0]                             */
#define HF_CUT_LEP_PT_MIN 3      /* pT(lepton 1) > params[0] GeV                           */
#define HF_CUT_MET_MIN 4         /* |MET| > params[0] GeV, after smearing                  */
#define HF_CUT_W_NU_SOLVABLE 5   /* W-mass neutrino p_z exists (Sect. 6.2)                 */
#define HF_CUT_HADTOP_CHI2_MAX 6 /* min over jet triplets of Eq. 1 hadronic chi2 < params[0] */
#define HF_CUT_LEP_OS 7          /* q1 * q2 < 0                                            */
#define HF_CUT_DILEP_SOLVABLE 8  /* >= 1 two-neutrino solution over b-jet pairings (Sect. 4) */
#define HF_CUT_HIGGS_WINDOW 9    /* params[0] < m_bb < params[1] (Sect. 4)                  */
#define HF_CUT_TTBAR_CHI2_MAX 10 /* full Eq. 1 fit (Sect. 6.2): min over the hadronic b-jet, the W
                                    jet pair, the leptonic b-jet and the neutrino p_z solution of
                                    the hadronic and leptonic top and W terms < params[0]; an
                                    analysis with it reports (m_top hadronic, m_top leptonic,
                                    chosen p_z, |MET|) and histograms the hadronic top mass */

typedef struct {
    int32_t kind;      /* HF_CUT_*                                                     */
    float params[4];   /* thresholds; integers for counts                              */
    uint32_t dep_mask; /* bit j: this cut must execute after user-order cut j           */
    uint8_t reorderable; /* 0 pins this cut to its user position for execution        */
    uint8_t pad[3];
} hf_cut;

typedef struct {
    int32_t event_model; /* HF_MODEL_*                                              */
    uint32_t n_cuts;     /* 1..16                                                    */
    const hf_cut* cuts;  /* host, n_cuts entries, USER order; copied by the call      */
    float mW, mt;        /* W and top masses, GeV (Sect. 4: 80.4, 172.5)              */
    float sigma_t, sigma_W; /* widths of Eq. 1, GeV                                  */
    float mH;            /* Higgs mass for the b-jet pair, GeV (Sect. 4: 125)          */
    float sigma_jet;     /* relative jet-energy resolution of the smearing, [0, 0.15]  */
    float sigma_met;     /* absolute MET resolution per component, GeV, >= 0           */
    uint32_t hist_nbins; /* reconstructed-mass histogram: bins, 1..1024                */
    float hist_lo, hist_hi; /* range, GeV; hist_lo < hist_hi                            */
    uint32_t record_levels; /* per-cut variable recording (Sect. 3): bit k records the
                               events that pass cuts 0..k (user order) in at least one
                               variation; 0 = no recording; bits >= n_cuts are invalid  */
    uint32_t record_vars[4]; /* HF_VAR_* stored in hf_record.value[0..3]               */
    float sigma_lep;     /* relative lepton-energy resolution of the smearing, [0, 0.15]:
                            lepton l of a unit is scaled by 1 + sigma_lep z[14 + l] (Sect. 4:
                            every measured object is smeared); with sigma_lep != 0 the lepton
                            pT cut and the W-mass solvability are decided per unit           */
    uint32_t per_event;  /* HF_PER_EVENT_*: what an event reports from its variations       */
} hf_analysis_desc;

/* hf_analysis_desc.per_event */
#define HF_PER_EVENT_MEAN 0u /* reco = mean over the surviving variations; the histogram is
                                filled once per surviving unit                               */
#define HF_PER_EVENT_BEST 1u /* best-of-variations (Sect. 4, ttH_sci: of the pseudo-experiments
                                only the most probable solution is kept): reco = the quantities
                                of the surviving variation with the smallest fit score -- the
                                hadronic chi2 of Eq. 1, the full Eq. 1 chi2 with the full fit,
                                m_ttbar of the chosen solution in the dilepton model -- ties to
                                the lowest variation; hf_results.best_v receives it; the
                                histogram is filled once per selected event with that
                                variation's value.  Device-resident single runs, the
                                allocation-free run and unbatched submissions; not the plain
                                form, hf_run_batch, HF_FLAG_BATCHING or together with per-cut
                                records (HF_EINVAL)                                           */

/* Variables of the per-cut recording.  A variable is stored at every
 * recorded level; where it is not defined yet at that level it holds its
 * default, 0 (Sect. 3: variables not yet updated keep their default). */
#define HF_VAR_NONE 0u    /* always 0                                                    */
#define HF_VAR_NJETS 1u   /* number of jets                                              */
#define HF_VAR_NBTAG 2u   /* number of b-tagged jets                                     */
#define HF_VAR_LEP_PT 3u  /* pT of the event's first lepton, GeV (FP64, rounded to float) */
#define HF_VAR_MET 4u     /* |MET| as measured (not smeared), GeV (FP64, rounded to float) */
#define HF_VAR_RECO0 5u   /* hf_results.reco[0..3] (+0..3): defined at the last cut only */
#define HF_VAR_RECO3 8u

/* One record: event (index within the chunk) e passes cuts 0..level in at
 * least one variation.  24 bytes. */
typedef struct {
    uint32_t event;
    uint32_t level;
    float value[4];
} hf_record;

/* Validates and registers an analysis.  *analysis_id receives its id.
 * Errors: HF_EINVAL (unknown kind, n_cuts out of range, missing
 * reconstruction cut for the model, dependency cycle, bad widths/histogram). */
hf_status hf_define_cuts(hf_ctx* ctx, const hf_analysis_desc* desc, uint32_t* analysis_id);

/* ------------------------------------------------------------------ */
/* Event columns (structure of arrays, one chunk of N events).          */
/* ------------------------------------------------------------------ */
typedef struct {
    const uint32_t* jet_off; /* N+1 offsets into jets; jet_off[0] = 0; n_jets <= 12   */
    const float* jets;       /* 4*J floats: (px, py, pz, E) per jet, GeV, 16-byte aligned */
    const uint16_t* btag;    /* N: bit i <=> jet i of the event is b-tagged          */
    const float* lep;        /* 4*L*N floats: (px, py, pz, E) of L leptons per event  */
    const int8_t* lep_q;     /* L*N charges                                         */
    const float* met;        /* 2*N floats: MET (x, y), GeV                           */
    uint64_t n_jets_total;   /* J = jet_off[N]                                       */
} hf_columns;

/* Results; every pointer may be NULL to skip that field. */
typedef struct {
    uint8_t* mask;      /* N: 1 if at least one variation of the event passed every cut */
    uint64_t* cutflow;  /* n_cuts+1, user order: [0] = units in, [k] = units passing cuts 1..k */
    uint64_t* hist;     /* hist_nbins+2: [0] underflow, [1..nbins] bins, [nbins+1] overflow  */
    uint16_t* n_surv;   /* N: variations of the event passing every cut                  */
    float* reco;        /* 4*N: per-event mean over passing variations, summed in variation
                           order; semileptonic (m_top, m_W, pz_nu, |MET|) -- with the full
                           fit (m_top had, m_top lep, pz_nu, |MET|) --, dilepton
                           (m_bb, m_t, m_tbar, m_ttbar); zeros when n_surv = 0           */
    uint64_t* recheck_count; /* 1: units re-evaluated in FP64 (diagnostic)              */
    hf_record* records; /* per-cut records of an analysis with record_levels != 0, in
                           (event, level) order; device memory (the device-resident entry
                           points only: hf_fetch_results rejects it)                      */
    uint64_t record_cap; /* records entries; records beyond it are counted, not written */
    uint64_t* n_records; /* 1 (device): records produced (may exceed record_cap)         */
    uint16_t* best_v;    /* N: with HF_PER_EVENT_BEST, the chosen variation (0xffff without a
                            surviving one); ignored otherwise                                */
} hf_results;

/* Asynchronous chunk submission (the serving entry point): a chunk of events
 * read by the caller enters the pipeline while earlier chunks are processed
 * (Sect. 5.1: input reading and event processing run simultaneously; the
 * events of a chunk are independent and processed in parallel).  Admission: the
 * chunk's device bytes (columns, results and cut-flow state, which stay
 * device-resident until fetched) must fit the context's HBM budget next to
 * the chunks in flight, else HF_EBUSY (nothing enqueued; retry after a fetch).
 * The columns are copied on the context's host-to-device stream, overlapping
 * the chunks already computing.  Without HF_FLAG_BATCHING the chunk's run is
 * enqueued at once on the compute stream; with it the chunk is QUEUED until
 * the dispatcher launches it in the next batch.  host_cols are HOST pointers, caller-owned,
 * that must stay valid and unchanged until the ticket is DONE or FAILED
 * (the library copies them to the device, from pinned memory directly or via
 * its pinned staging).  first_event_id is the global id of event 0 (it keys
 * the smearing); seed keys the smearing; n_variations = V in 1..HF_MAX_VARIATIONS.
 * *ticket receives the ticket.  Errors: HF_EINVAL (bad columns or sizes),
 * HF_ENOTFOUND (analysis), HF_EBUSY (budget or slots; nothing enqueued),
 * HF_ENOMEM, HF_ECUDA.  Malformed offsets or n_jets > 12 found on the device
 * make the ticket FAILED with HF_EINVAL at fetch. */
hf_status hf_submit_chunk(hf_ctx* ctx, uint32_t analysis_id, const hf_columns* host_cols,
                          uint64_t n_events, uint64_t first_event_id, uint64_t seed,
                          uint32_t n_variations, uint64_t* ticket);

#define HF_STATE_QUEUED 0
#define HF_STATE_RUNNING 1
#define HF_STATE_DONE 2
#define HF_STATE_FAILED 3

/* Non-blocking state query of a ticket (the chunk's place in the pipeline of
 * Sect. 5.1).  Errors: HF_ENOTFOUND. */
hf_status hf_poll(hf_ctx* ctx, uint64_t ticket, int32_t* state);

/* The outputs of a chunk (Sect. 3: the selected events, the per-cut counts
 * and the user's histograms; Appendix I: histogram filling).  Waits (bounded
 * by timeout_ms; 0 = poll once) for the ticket, then copies its
 * results into the caller's HOST buffers of `out` (NULL fields skipped) and
 * releases the ticket.  Errors: HF_ETIMEOUT (ticket kept), HF_ENOTFOUND,
 * HF_EINVAL (device found malformed columns; ticket released), HF_ECUDA. */
hf_status hf_fetch_results(hf_ctx* ctx, uint64_t ticket, hf_results* out, uint32_t timeout_ms);

/* Synchronous-on-stream run over DEVICE-resident columns: enqueues the whole
 * path on `stream` (cudaStream_t, NULL = the context's stream) and writes the
 * results into DEVICE buffers of `dev_out` (NULL fields skipped; cutflow and
 * hist are overwritten, not accumulated).  Scratch memory is owned by the
 * context and reused; calls on one context are serialised by its mutex, and
 * results are valid once the stream reaches them.  n_events may be 0.
 * Errors: HF_EINVAL, HF_ENOTFOUND, HF_ENOMEM, HF_ECUDA.  Malformed columns set
 * the error word readable with hf_device_error. */
hf_status hf_run_device(hf_ctx* ctx, uint32_t analysis_id, const hf_columns* dev_cols,
                        uint64_t n_events, uint64_t first_event_id, uint64_t seed,
                        uint32_t n_variations, const hf_results* dev_out, void* stream);

/* Same as hf_run_device with the plain form: one thread per event, cuts in user
 * order, jets read from global memory, no compaction, staging or reordering.
 * Identical results (same FP32 bands and FP64 recheck); the comparison baseline. */
hf_status hf_run_device_plain(hf_ctx* ctx, uint32_t analysis_id, const hf_columns* dev_cols,
                              uint64_t n_events, uint64_t first_event_id, uint64_t seed,
                              uint32_t n_variations, const hf_results* dev_out, void* stream);

/* ------------------------------------------------------------------ */
/* Batched runs: many chunks through one fixed launch sequence.         */
/* ------------------------------------------------------------------ */
/* One chunk of a batch: its analysis, smearing keys, DEVICE columns and
 * DEVICE result buffers (caller-owned; NULL result fields are skipped, the
 * cut flow and histogram are overwritten, not accumulated). */
typedef struct {
    uint32_t analysis_id;    /* registered analysis, either event model               */
    uint32_t n_variations;   /* V in 1..HF_MAX_VARIATIONS                              */
    uint64_t n_events;       /* N < 2^32 (0 allowed)                                   */
    uint64_t first_event_id; /* global id of event 0 (keys the smearing)               */
    uint64_t seed;           /* smearing seed                                          */
    hf_columns cols;         /* DEVICE columns, layout as for hf_run_device            */
    hf_results out;          /* DEVICE results of this chunk                           */
} hf_chunk;

/* Runs n_chunks chunks of uneven size -- any mix of analyses (hence of the
 * semileptonic and dilepton models), sizes and variation counts -- on
 * `stream` (NULL = the context's stream) through one fixed sequence of
 * persistent kernels: a column scan and compaction over all chunks, one
 * stage-2 grid per jet multiplicity (and one for the dilepton model) that
 * takes tiles of every chunk from a device work queue, and one FP64 recheck
 * (Sect. 3: every chunk's events pass the ordered cut chain; Sect. 5: many
 * independent event sets processed concurrently).  The sequence does not
 * depend on the number of chunks; the context captures it once as a CUDA
 * graph and replays the graph for later batches that fit the same scratch
 * layout.  Each chunk's results equal those of hf_run_device on that chunk.
 * Cut execution orders are each analysis's current ones; the scheduler
 * updates each analysis once after the batch from the batch's statistics.
 * chunks: HOST array (copied by the call).  The context's scratch arena is
 * grown as needed (device allocation outside any stream capture).
 * Errors: HF_EINVAL (a chunk's sizes, pointers or V), HF_ENOTFOUND (analysis),
 * HF_ENOMEM, HF_ECUDA.  Malformed columns set the device error word. */
hf_status hf_run_batch(hf_ctx* ctx, const hf_chunk* chunks, uint32_t n_chunks, void* stream);

/* Autotuner of the stage-2 tile shape: runs the fast path on a sample of
 * DEVICE columns (n_events >= 1, typically 10^5..10^6 events of the workload)
 * with each candidate number of units per tile (semileptonic 128, 256, 512,
 * 1024; dilepton 32, 64, 128, 256), timed with CUDA events on the context's
 * stream after a warm-up run, and keeps the fastest for this analysis's event
 * model and the variation class of n_variations (V = 1, 2-3, 4-7, ..., >= 128)
 * in the context; later hf_run_device, hf_submit_chunk and hf_run_batch
 * calls with that model and class use it.  *units_per_tile (may be NULL)
 * receives the choice.  Synchronises the context's stream.
 * Errors: HF_EINVAL, HF_ENOTFOUND, HF_ENOMEM, HF_ECUDA. */
hf_status hf_autotune(hf_ctx* ctx, uint32_t analysis_id, const hf_columns* dev_cols, uint64_t n_events,
                      uint32_t n_variations, uint64_t seed, int32_t* units_per_tile);

/* Waits for the context's stream and returns the device error word of the
 * last hf_run_device* or hf_run_batch call in *word (0 = none).  Bit 0: malformed
 * offsets or n_jets > 12 (those events get zero results).  Bit 1: the FP64-recheck list
 * of the run was full; the units that did not fit were re-evaluated in FP64 inside the
 * stage-2 kernels instead, so the results are still exact, only slower (diagnostic, not
 * an error of the results).  Bit 2: a bounded wait of a kernel on its
 * own asynchronous copies ran out (the run's results are then incomplete).
 * Errors: HF_ECUDA. */
hf_status hf_device_error(hf_ctx* ctx, uint32_t* word);

/* Scheduler state of an analysis: current execution order of its cuts
 * (user indices, n_cuts entries) and per-cut statistics accumulated so far
 * (units evaluated, units passed, summed cost in SM cycles).  Any pointer may
 * be NULL.  Synchronises the context's stream.  Errors: HF_ENOTFOUND. */
hf_status hf_sched_state(hf_ctx* ctx, uint32_t analysis_id, int32_t* exec_order,
                         uint64_t* evaluated, uint64_t* passed, uint64_t* cost);

/* Forces the execution order of an analysis's cuts (user indices); it must
 * respect dependencies.  Disables automatic reordering for that analysis.
 * Used to check that results do not depend on execution order.
 * Errors: HF_EINVAL (not a valid dependency-respecting permutation). */
hf_status hf_set_exec_order(hf_ctx* ctx, uint32_t analysis_id, const int32_t* exec_order);

/* Per-phase device time and work counters of the runs since the last reset,
 * collected when the context was opened with HF_FLAG_PROFILE.  Times come from
 * CUDA events recorded on the launching stream around each phase of the fast
 * path: stage 1 (multiplicity count, column cuts, compaction), stage 2 (the
 * per-multiplicity reconstruction kernels) and the FP64 recheck. */
#define HF_FLAG_PROFILE 8u
typedef struct {
    uint64_t runs;            /* fast-path runs profiled                            */
    double ms_stage1;         /* summed device time of stage 1, ms                  */
    double ms_stage2;         /* summed device time of stage 2, ms                  */
    double ms_recheck;        /* summed device time of the FP64 recheck, ms         */
    uint64_t launches_stage2; /* stage-2 kernel launches                            */
    uint64_t units_stage2;    /* units (event x variation) evaluated in stage 2     */
    uint64_t events_stage2;   /* events that reached stage 2                        */
    uint64_t units_top[16];   /* units that evaluated the triplet chi2, by n_jets   */
    uint64_t units_dilep[16]; /* units that evaluated the two-neutrino solve, by n_b */
    uint64_t pairings_dilep;  /* b-jet pairings solved                               */
    uint64_t cands_top;       /* triplet candidates evaluated                        */
    uint64_t batches;         /* batches launched by the dispatcher (HF_FLAG_BATCHING) */
    uint64_t batched_chunks;  /* chunks in those batches                             */
} hf_profile_data;

/* Waits for the profiled runs, writes the totals into *out (host) and, if
 * reset != 0, clears them.  Errors: HF_ESTATE (profiling not enabled), HF_ECUDA. */
hf_status hf_profile(hf_ctx* ctx, hf_profile_data* out, int32_t reset);

/* ------------------------------------------------------------------ */
/* HL-LHC multi-region top selection (Sect. 6.1).                       */
/* ------------------------------------------------------------------ */
/* Event columns of the selection (structure of arrays, one chunk of N
 * events; J jets and L leptons in total).  DEVICE memory for hf_run_hl. */
#define HF_HL_MAX_JETS 16u    /* jets per event (b-tag bits are 16 wide)          */
#define HF_HL_MAX_LEPTONS 4u  /* leptons per event                                 */
typedef struct {
    const uint32_t* jet_off;  /* N+1 offsets into jets; jet_off[0] = 0              */
    const float* jets;        /* 4*J floats (px, py, pz, E), GeV, 16-byte aligned     */
    const uint16_t* btag;     /* N: bit i <=> jet i of the event is b-tagged          */
    const uint32_t* lep_off;  /* N+1 offsets into the lepton columns; lep_off[0] = 0  */
    const float* lep;         /* 4*L floats (px, py, pz, E), 16-byte aligned          */
    const int8_t* lep_q;      /* L charges (+1 / -1)                                  */
    const uint8_t* lep_flav;  /* L flavours (0 electron, 1 muon)                      */
    const float* met;         /* 2*N floats: MET (x, y), GeV, 8-byte aligned           */
    uint64_t n_jets_total;    /* J = jet_off[N]                                       */
    uint64_t n_leptons_total; /* L = lep_off[N]                                       */
} hf_hl_columns;

/* Parameters of the selection (Sect. 6.1 values in brackets). */
typedef struct {
    float met_min;     /* every signal bin: |MET'| > met_min [30 GeV]                         */
    float mll_min;     /* ttbar 2l: M_ll > mll_min [40 GeV]                                    */
    float mtw_min;     /* Wt 1l: M_T^W > mtw_min [50 GeV]                                      */
    float dr_iso;      /* a lepton is isolated when no jet lies within Delta R < dr_iso [0.4] */
    float eta_bounds[3]; /* regions I |eta| < b0, II b0 < |eta| < b1, III b1 < |eta| < b2
                            [2.5, 2.75, 3.5]; 0 < b0 < b1 < b2                               */
    float sigma_met;   /* MET resolution per component of the variations, GeV, >= 0        */
    uint32_t hist_nbins; /* per-channel histograms of the leading isolated lepton pT, 1..1024 */
    float hist_lo, hist_hi;
} hf_hl_desc;

/* Channel codes. */
#define HF_HL_NONE 0
#define HF_HL_TTBAR_1L 1
#define HF_HL_TTBAR_2L 2
#define HF_HL_T_CHANNEL 3
#define HF_HL_WT_1L 4
#define HF_HL_WT_2L 5

/* DEVICE result buffers, caller-owned; NULL fields are skipped. */
typedef struct {
    uint64_t* counts;  /* 6: units per channel code (HF_HL_*), overwritten              */
    uint64_t* hist;    /* 5 * (hist_nbins + 2): channel c (1..5) at (c - 1) * (nbins + 2):
                          [0] underflow, [1..nbins], [nbins + 1] overflow; overwritten      */
    int8_t* channel;   /* N * V: channel code of unit (event e, variation v) at e * V + v  */
} hf_hl_results;

/* The HL-LHC multi-region top selection (Sect. 6.1) over DEVICE-resident
 * columns, enqueued on `stream` (NULL = the context's stream).  Per unit
 * (event, variation v < n_variations): the jets' pseudorapidity regions (a
 * boundary, or |eta| >= b2, in none), b-jets = b-tagged jets of region I,
 * isolated leptons (no jet within Delta R < dr_iso; Delta R^2 = Delta eta^2 +
 * Delta phi^2, Delta phi wrapped to [-pi, pi]), then, with |MET'| > met_min:
 * one isolated lepton -- ttbar 1l (>= 4 jets in I, exactly 2 b, none in II or
 * III), t-channel (exactly 1 jet in I and exactly 1 in II or III, exactly 1
 * b), Wt 1l (exactly 3 jets in I, exactly 1 b, none in II or III, M_T^W >
 * mtw_min, M_T^W^2 = 2 (pT |MET'| - pT . MET')); two isolated leptons of
 * opposite sign and different flavour -- ttbar 2l (>= 2 jets in I, exactly
 * 2 b, none in II or III, M_ll > mll_min), Wt 2l (1 or 2 jets in I, exactly
 * 1 b, none in II or III); otherwise none.  The variations smear MET only:
 * MET' = MET + sigma_met (z12, z13), the unit's Philox normals keyed by
 * (seed, first_event_id + e, v) as in the other event models.  A unit in a
 * signal channel adds one entry at the leading isolated lepton's pT to that
 * channel's histogram.  Every decision equals the FP64 definition's
 * (FP32 with error bands, FP64 inside them).  n_events < 2^32, may be 0.
 * Errors: HF_EINVAL (NULL or misaligned pointers, bad parameters),
 * HF_ENOMEM, HF_ECUDA.  Events with malformed offsets, more than
 * HF_HL_MAX_JETS jets or HF_HL_MAX_LEPTONS leptons set bit 0 of the device
 * error word (hf_device_error), get channel 0 and are not counted. */
hf_status hf_run_hl(hf_ctx* ctx, const hf_hl_desc* desc, const hf_hl_columns* dev_cols, uint64_t n_events,
                    uint64_t first_event_id, uint64_t seed, uint32_t n_variations, const hf_hl_results* dev_out,
                    void* stream);

/* ------------------------------------------------------------------ */
/* Measurement.                                                         */
/* ------------------------------------------------------------------ */
/* Measured FP32 throughput of the device, the denominator of the FP32
 * roofline of the reconstruction kernels (the paper has no counterpart; it
 * reports no absolute rates).  Runs a full grid of independent fused
 * multiply-add chains for about a second in total -- scalar fmaf and the
 * packed two-lane fma.rn.f32x2 of sm_100 and later -- timed with CUDA events
 * on a private stream after a warm-up launch, and writes the best of three
 * timed launches of each (2 flops per lane per fma) and the SM count into
 * *out (host).  Allocates and frees a few KB of device memory; restores the
 * calling thread's current device.  Errors: HF_EINVAL (NULL out, bad
 * device), HF_ECUDA. */
typedef struct {
    int32_t sm_count;     /* multiprocessors of the device                     */
    double tflops_ffma;   /* scalar FFMA, TFLOP/s                              */
    double tflops_ffma2;  /* packed two-lane FFMA, TFLOP/s                     */
} hf_fp32_peak_result;
hf_status hf_fp32_peak(int32_t device, hf_fp32_peak_result* out);

/* ------------------------------------------------------------------ */
/* Allocation-free run.                                                 */
/* ------------------------------------------------------------------ */
/* The paper has no counterpart of this entry point: it serves callers that
 * cannot allocate device memory when they run a chunk -- code inside a CUDA
 * stream capture, plug-ins of frameworks that own every device allocation,
 * real-time loops that must not allocate.  It runs the same path as
 * hf_run_device (same results; cuts executed in user order, no scheduler)
 * without a context and without allocating: no cudaMalloc, cudaFree or other
 * allocating call.  Its scratch memory is one static device array of
 * HF_NOALLOC_SCRATCH_BYTES in the library, which every GPU that loads the
 * library holds until the process exits.
 *   - Without a context there is no device error word to read: events with
 *     malformed offsets or more than 12 jets get zero results (mask 0,
 *     n_surv 0, reco 0, and no entry in the cut flow, not even cutflow[0])
 *     and the call still returns HF_OK.  Callers that need malformed columns reported run
 *     hf_run_device on them.  The FP64-recheck list of the array holds 65,536
 *     units; beyond that the units are re-evaluated in FP64 inside the stage-2
 *     kernels (same results, slower).
 *   - desc, dev_cols, dev_out, stream: as for hf_define_cuts and
 *     hf_run_device (DEVICE column and result buffers, caller-owned; NULL
 *     result fields are skipped; stream NULL = the legacy default stream).
 *   - n_events <= HF_NOALLOC_MAX_EVENTS, else HF_EINVAL with a message.
 *   - The first call on a device looks up the array's device address on that
 *     device (current device at the call); make that first call before any
 *     stream capture.  After a cudaDeviceReset the next call on that device
 *     finds the old address stale and looks it up again: it counts as a first
 *     call.
 *   - Every call shares the one array and clears its counters at the start;
 *     calls whose work overlaps on the GPU (different streams, or several
 *     host threads without ordering) race and give wrong results: order them.
 * Errors: HF_EINVAL, HF_ECUDA. */
#define HF_NOALLOC_MAX_EVENTS 1048576u
#define HF_NOALLOC_SCRATCH_BYTES 15508736u
hf_status hf_run_device_noalloc(const hf_analysis_desc* desc, const hf_columns* dev_cols, uint64_t n_events,
                                uint64_t first_event_id, uint64_t seed, uint32_t n_variations,
                                const hf_results* dev_out, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* HF_H */
