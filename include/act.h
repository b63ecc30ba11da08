/*
 * act.h -- C ABI of the GB300 residual-projection matching-pursuit library
 * for Gaussian-chirplet dictionaries (Adaptive Chirplet Transform).
 *
 * The operation (Sec. III-A, Eq. (3)-(4), Fig. 1): given real signals s and a
 * finite grid of chirplet parameters theta = (tc, fc, logDt, c), return P
 * atoms theta_k with coefficients c_k and the residual r_P of the greedy
 * decomposition
 *     r_0 = s;  i* = argmax_i |<g_i, r_k>|;  c_k = <g*, r_k>;
 *     r_{k+1} = r_k - c_k g*,
 * where every g_i is the real part of Eq. (1) sampled on the window and
 * scaled to unit l2 norm (Sec. III-A).  The projection of all atoms against
 * the residual is the matrix product P = D X^T of Sec. IV-A; the BFGS
 * refinement of Fig. 1 is not part of this library's search.
 *
 * Units: tc in samples (0 = first sample), tau = (n - tc) / fs seconds,
 * fc in Hz, c in Hz/s multiplying tau^2 in the phase of Eq. (1) (the
 * instantaneous frequency is fc + 2 c tau), Dt = exp(logDt) seconds.
 * Flat atom index: ((i_tc * N_fc + i_fc) * N_logDt + i_logDt) * N_c + i_c.
 * Ties in |score| go to the lowest flat index.
 *
 * Conventions for every call:
 *   - no call throws; each returns an act_status;
 *   - the library owns the grid, its dictionary and all work buffers; the
 *     caller owns every signal and output buffer it passes in;
 *   - input buffers are never modified;
 *   - calls that take a cuda_stream (a cudaStream_t, NULL = legacy default
 *     stream) enqueue their GPU work on it and return without waiting,
 *     except where a host buffer forces a copy back (then they wait);
 *   - a grid may be used by one host thread at a time, and its calls share
 *     the grid's work buffers: calls on different streams must be ordered
 *     (an event or a synchronisation between them), or they overwrite each
 *     other's residuals and results.
 */
#ifndef ACT_H
#define ACT_H

#include <stdint.h>

#if defined(__GNUC__)
#define ACT_API __attribute__((visibility("default")))
#else
#define ACT_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    ACT_OK = 0,
    ACT_ERR_INVALID_ARG = 1,    /* NULL pointer, bad size, bad grid */
    ACT_ERR_OOM = 2,            /* device allocation failed (no CPU fallback) */
    ACT_ERR_CUDA = 3,           /* a CUDA runtime call failed */
    ACT_ERR_NONFINITE = 4,      /* an input signal held NaN or Inf */
    ACT_ERR_DEVICE_TIMEOUT = 5, /* a bounded device-side wait gave up */
    ACT_ERR_NOT_BUILT = 6,      /* act_dictionary_build has not run */
    ACT_ERR_UNSUPPORTED = 7     /* size or mode outside what the library handles */
} act_status;

/* One grid axis: value_i = lo + i * step, i = 0 .. count-1. */
typedef struct {
    double lo;
    double step;
    int32_t count;
} act_axis;

/* A dictionary grid (Sec. III-A, Table 2) on an n_samples window at fs Hz. */
typedef struct {
    int32_t n_samples; /* window length L, 1 .. 2048 */
    double fs;         /* sample rate, Hz */
    act_axis tc;       /* time centre, samples */
    act_axis fc;       /* frequency centre, Hz */
    act_axis logdt;    /* natural log of the duration in seconds */
    act_axis c;        /* chirp rate, Hz/s */
} act_grid_desc;

/* How act_dictionary_build stores the dictionary.
 *   ACT_DICT_FP32: D as FP32 [K][Lp] (Lp = L rounded up to 128), searched by
 *                  the FP32 GEMV / multi-channel GEMV.
 *   ACT_DICT_BF16: D as FP32 [K][Lp] plus BF16 [K][Lb] (Lb = L rounded up to
 *                  64) for the tensor-core search; FP32 rows are used to
 *                  rescore candidates and for the update.
 *   ACT_DICT_AUTO: ACT_DICT_FP32 when the FP32 rows fit the grid's memory
 *                  budget (act_set_memory_budget; by default 90% of the
 *                  device memory free when the build starts), otherwise
 *                  ACT_DICT_RECOMPUTE when the time centres are whole
 *                  samples and the templates fit; otherwise the build
 *                  returns ACT_ERR_OOM and keeps nothing (a grid with
 *                  fractional time centres has no template form: its only
 *                  search without stored rows is ACT_SEARCH_LEM).
 *                  act_dictionary_mode reports the choice.
 *   ACT_DICT_RECOMPUTE: no atom rows are stored.  The real atom of Eq. (1)
 *                  depends on n and tc only through n - tc, so on a grid
 *                  whose time centres are whole samples (tc.lo and tc.step
 *                  integers, step >= 1) every atom is a window of one
 *                  template per (fc, logDt, c).  The build stores those
 *                  templates (FP32, the lags the window can see) and one FP32
 *                  scale 1/|u| per atom; the search (ACT_SEARCH_SHIFT) forms
 *                  every atom's samples in-kernel from its template and scores
 *                  all time centres of a template as one cross-correlation.
 *                  Memory: about (N_fc N_logDt N_c)(S + 1)(ceil(L/S) + N_tc)
 *                  x 4 bytes instead of K x L x 4 (S = tc.step). */
typedef enum {
    ACT_DICT_AUTO = 0,
    ACT_DICT_FP32 = 1,
    ACT_DICT_BF16 = 2,
    ACT_DICT_RECOMPUTE = 3
} act_dict_mode;

/* Which search act_decompose runs.
 *   ACT_SEARCH_FP32: FP32 GEMV with the argmax fused (CUDA cores).
 *   ACT_SEARCH_BF16: BF16 tcgen05 GEMM over all atoms (tensor cores, FP32
 *                    accumulation) reduced to the largest |score| per
 *                    tile and per 32-atom block; the blocks that an error
 *                    bound cannot exclude are rescored in FP32 (a channel
 *                    with more than 512 of them takes the FP32 search), so
 *                    the selection equals the FP32 search's bit for bit
 *                    (any number of channels, in tiles of 128).
 *   ACT_SEARCH_LEM:  the hierarchical search of act_lem_params (no
 *                    dictionary needed; act_atom.flat_index is -1).
 *   ACT_SEARCH_SHIFT: the template search over an ACT_DICT_RECOMPUTE build
 *                    (FP32 CUDA cores, every atom scored, the selected atom
 *                    read back from its template for the update).
 *   ACT_SEARCH_SHIFT_BF16: the same selection on tensor cores: BF16
 *                    templates x shifted BF16 residual rows (tcgen05, FP32
 *                    accumulation, every score scaled by its atom's 1/|u|)
 *                    reduced to the largest |score| per (time centre,
 *                    32-template block); the blocks an error bound cannot
 *                    exclude are rescored with ACT_SEARCH_SHIFT's own
 *                    arithmetic (a channel with more than 1,024 of them is
 *                    searched by ACT_SEARCH_SHIFT in full), so the selection
 *                    equals ACT_SEARCH_SHIFT's bit for bit.
 *   ACT_SEARCH_AUTO: BF16 when the dictionary was built with ACT_DICT_BF16,
 *                    SHIFT_BF16 with ACT_DICT_RECOMPUTE (SHIFT where the
 *                    tensor-core view could not be set up), FP32 otherwise. */
typedef enum {
    ACT_SEARCH_AUTO = 0,
    ACT_SEARCH_FP32 = 1,
    ACT_SEARCH_BF16 = 2,
    ACT_SEARCH_LEM = 3,
    ACT_SEARCH_SHIFT = 4,
    ACT_SEARCH_SHIFT_BF16 = 5
} act_search_mode;

/* Settings of the LEM-inspired hierarchical search (Sec. VII-A, Fig. 7),
 * which needs no stored dictionary: per order, a Latin hypercube sample of
 * n_coarse parameter vectors over the grid's box (0: as many as the coarse
 * grid of steps[0] would hold, at most 16384), the top_k by |<g, r_k>| kept;
 * then for each of `levels` refinement levels (0..2) the neighbourhood
 * dictionary of every kept candidate -- offsets of -radius..radius steps of
 * that level's steps per axis, clamped to the box -- pooled and reranked to
 * a new top_k (1..16); the best candidate starts the BFGS refinement
 * (act_set_refinement; 0 iterations keeps it as is).  Axes in the order
 * (tc [samples], fc [Hz], logDt, c [Hz/s]).  The draws come from SplitMix64
 * seeded with `seed` (counter = channel, order, axis, draw). */
typedef struct {
    int32_t n_coarse;
    int32_t top_k;
    int32_t levels;
    double steps[3][4];
    int32_t radius[4];
    uint64_t seed;
} act_lem_params;

/* One selected atom: its grid parameters and flat index. */
typedef struct {
    double tc;
    double fc;
    double logdt;
    double c;
    int64_t flat_index;
} act_atom;

typedef struct act_grid act_grid; /* opaque, library-owned */

/* Human-readable name of a status code (static string, never NULL). */
ACT_API const char *act_status_string(act_status status);

/* Detail of the last failing CUDA call made by this library on the calling
 * host thread ("" when none); valid until the next call on that thread. */
ACT_API const char *act_last_error_message(void);

/* Fills *out from (start, stop, step) triples enumerated as half-open
 * sequences start, start+step, ... < stop, which is how the ranges of
 * Table 2 give their printed combination counts.  Host only, no GPU.
 * Errors: ACT_ERR_INVALID_ARG for NULL pointers, step <= 0, an empty axis,
 * n_samples outside 1..2048 or fs <= 0. */
ACT_API act_status act_grid_from_ranges(int32_t n_samples, double fs, const double tc[3],
                                const double fc[3], const double logdt[3], const double c[3],
                                act_grid_desc *out);

/* Creates a grid on CUDA device `device` (Sec. III-A).  Allocates nothing
 * large: the dictionary is made by act_dictionary_build.  *out receives the
 * handle.  Errors: ACT_ERR_INVALID_ARG (bad descriptor, more than 2^32-1
 * atoms), ACT_ERR_CUDA (device not usable). */
ACT_API act_status act_grid_create(const act_grid_desc *desc, int32_t device, act_grid **out);

/* Number of atoms K of the grid and the FP32 row stride Lp in floats. */
ACT_API act_status act_grid_size(const act_grid *grid, int64_t *n_atoms, int32_t *row_stride);

/* Generates every atom on the device (Eq. (1) real part, unit l2 norm,
 * Sec. III-A) in the layout `mode` selects, replacing any earlier build.
 * Enqueued on cuda_stream.  Errors: ACT_ERR_OOM when the dictionary does not
 * fit (nothing is kept), ACT_ERR_UNSUPPORTED for ACT_DICT_RECOMPUTE on a grid
 * whose time centres are not whole samples. */
ACT_API act_status act_dictionary_build(act_grid *grid, act_dict_mode mode, void *cuda_stream);

/* The dictionary the last successful act_dictionary_build made
 * (ACT_DICT_FP32, ACT_DICT_BF16 or ACT_DICT_RECOMPUTE; an ACT_DICT_AUTO build
 * reports what it chose) into *mode.  ACT_ERR_NOT_BUILT (and *mode = -1)
 * when there is none. */
ACT_API act_status act_dictionary_mode(const act_grid *grid, int32_t *mode);

/* Device bytes an ACT_DICT_AUTO build may give the dictionary (0, the
 * default: 90% of the device memory free when the build starts). */
ACT_API act_status act_set_memory_budget(act_grid *grid, uint64_t bytes);

/* Limit, in nanoseconds, of every bounded device-side wait in this grid's
 * kernels (a pipeline stage waiting for its copy or its consumer).  A wait
 * that reaches it gives up: the kernel records ACT_ERR_DEVICE_TIMEOUT for
 * act_grid_status, lets the copies it already issued land, releases its
 * tensor memory and exits, leaving the context usable; that decomposition's
 * outputs are then not valid.  Default 2,000,000,000 (2 s).  0 gives up at
 * the first unsuccessful poll (used to test the timeout path).  Errors:
 * ACT_ERR_INVALID_ARG for ns < 0.  Changing it re-records the grid's graphs
 * and makes ragged plans built on the grid stale. */
ACT_API act_status act_set_wait_limit(act_grid *grid, int64_t ns);

/* Whether the tensor-core template search (ACT_SEARCH_SHIFT_BF16) may run
 * its GEMM on CTA pairs: a cluster of two CTAs on two SMs shares each
 * tcgen05 MMA (cta_group::2, M = 256: each CTA's 128 shifted residual rows
 * against one 256-template tile), each SM staging its own rows and half of
 * the templates.  1 (the default): pairs where they apply (256-template
 * tiles, at least two row tiles, a work unit for every pair the device
 * holds); 0: one SM per MMA (M = 128) always.  Selections are identical
 * either way.  Errors: ACT_ERR_INVALID_ARG for other values.  Changing it
 * re-records the grid's graphs. */
ACT_API act_status act_set_cta_pairs(act_grid *grid, int32_t enable);

/* *used = 1 when a `channels`-channel ACT_SEARCH_SHIFT_BF16 decomposition on
 * this grid (as built and set now) runs its GEMM on CTA pairs, else 0
 * (also without a template build).  Errors: ACT_ERR_INVALID_ARG for
 * channels < 1 or a null pointer. */
ACT_API act_status act_get_cta_pairs(const act_grid *grid, int32_t channels, int32_t *used);

/* Single-launch decomposition (Fig. 1's loop: search, selection and the
 * Eq. (4) update for every order) over a small stored FP32 dictionary.
 * Where it applies (the FP32 search over an ACT_DICT_FP32 dictionary of at
 * most 512 MiB; one or two channels; no refinement; the
 * grid not profiling; a device that runs cooperative launches) every
 * act_decompose is one cooperative kernel: each CTA scores its share of
 * the rows against its own shared-memory copy of the residuals, a bounded
 * grid barrier per order makes the winners known, and every CTA applies
 * the update to its copy.  The results are bit for bit those of the
 * per-order GEMV and update kernels; the launch latency of 2P dependent
 * kernels is what it saves.  With every buffer in device memory the call
 * is one memset and that launch (no graph, no copies); with host buffers
 * the launch runs inside the grid's graph, between the copies.  ctas_per_sm: CTAs per SM of that launch
 * (capped by how many fit), 0 = never use it; the default is 2.  Errors:
 * ACT_ERR_INVALID_ARG for values outside 0..32.  Changing it re-records
 * the grid's graphs.  A barrier wait that runs past the grid's wait limit
 * (act_set_wait_limit) makes the launch give up: the next synchronising
 * call returns ACT_ERR_DEVICE_TIMEOUT. */
ACT_API act_status act_set_fused(act_grid *grid, int32_t ctas_per_sm);

/* *ctas = the number of CTAs of the single-launch decomposition a
 * `channels`-channel act_decompose on this grid (as built and set now)
 * launches, or 0 when it takes the per-order kernels.  Errors:
 * ACT_ERR_INVALID_ARG for channels < 1 or a null pointer. */
ACT_API act_status act_get_fused(const act_grid *grid, int32_t channels, int32_t *ctas);

/* Test aid for out-of-memory handling: the nth device allocation made by
 * this library from now on (any grid, any thread; nth >= 1) fails once, as
 * if the device were out of memory.  The call that makes it returns
 * ACT_ERR_OOM, frees what it had made for itself and keeps the grid usable
 * (a failed dictionary build keeps no dictionary).  0 disarms it.  Errors:
 * ACT_ERR_INVALID_ARG for nth < 0. */
ACT_API act_status act_inject_alloc_failure(int32_t nth);

/* Sets the hierarchical search (ACT_SEARCH_LEM).  A new grid starts with the
 * settings the paper reports for EEG: top_k 4, 2 levels, steps
 * (64, 2, 2, 5), (32, 1, 1, 2.5), (16, 0.5, 0.5, 0.5), radius (2, 2, 1, 2),
 * n_coarse 0, seed 0.  Errors: ACT_ERR_INVALID_ARG (non-positive steps,
 * top_k or levels out of range), ACT_ERR_UNSUPPORTED (more than 16384 coarse
 * samples).  Makes ragged plans built on this grid stale. */
ACT_API act_status act_set_lem(act_grid *grid, const act_lem_params *params);

/* Selects the search act_decompose runs (see act_search_mode). */
ACT_API act_status act_set_search(act_grid *grid, act_search_mode mode);

/* Residual-projection matching pursuit (Eq. (4), Fig. 1) of `channels`
 * independent signals, n_atoms orders each, as one CUDA-graph launch.
 *   signals       [channels][n_samples] float32, device or host memory;
 *   atoms_out     [channels][n_atoms] act_atom, device or host, may be NULL;
 *   coeffs_out    [channels][n_atoms] float32 c_k, device or host, may be NULL;
 *   residuals_out [channels][n_samples] float32 r_P, device or host, may be NULL;
 *   energy_out    [channels][n_atoms+1] float64 |r_k|^2 for k = 0..n_atoms
 *                 (FP64 sums of the FP32 residual), device or host, may be NULL.
 * Device/host is detected per pointer.  With only device buffers the call
 * returns after enqueueing; with any host buffer it waits for the result.
 * Errors: ACT_ERR_NOT_BUILT, ACT_ERR_INVALID_ARG (channels < 1,
 * n_atoms < 1, NULL signals), ACT_ERR_OOM, ACT_ERR_CUDA.  A NaN/Inf in the
 * signals or a device-side timeout is reported by act_grid_status. */
ACT_API act_status act_decompose(act_grid *grid, const float *signals, int32_t channels, int32_t n_atoms,
                         act_atom *atoms_out, float *coeffs_out, float *residuals_out,
                         double *energy_out, void *cuda_stream);

/* Projection P = D X^T of Sec. IV-A without the selection: scores
 * [channels][K] float32 (device memory) of every atom against each of
 * `channels` signals [channels][n_samples] (device memory), on the FP32
 * dictionary or, for an ACT_DICT_RECOMPUTE build, by the template search.
 * Errors as act_decompose. */
ACT_API act_status act_project(act_grid *grid, const float *signals, int32_t channels, float *scores,
                       void *cuda_stream);

/* Copies `count` FP32 dictionary rows starting at atom `first` into
 * out[count][n_samples] (device or host memory); waits when out is host
 * memory.  ACT_ERR_UNSUPPORTED for an ACT_DICT_RECOMPUTE build (no rows). */
ACT_API act_status act_dictionary_rows(act_grid *grid, int64_t first, int64_t count, float *out,
                               void *cuda_stream);

/* Waits for cuda_stream and returns the first device-side error recorded
 * by this grid's kernels since the last call (ACT_ERR_NONFINITE,
 * ACT_ERR_DEVICE_TIMEOUT), then clears it; ACT_OK otherwise. */
ACT_API act_status act_grid_status(act_grid *grid, void *cuda_stream);

/* Off-grid refinement (Fig. 1: theta* = argmax_theta |<g(theta), r_k>|,
 * started from the grid winner; the paper runs BFGS on the CPU for it).
 * With steps > 0, every order's grid selection is followed on the GPU by
 * `steps` BFGS iterations per channel on -|<g(theta), r_k>| in coordinates
 * scaled by the grid steps (first step at most half a grid step, Armijo
 * backtracking, parameters kept inside the grid box widened by one step),
 * and the refined atom g(theta*), generated on the fly and unit-normalised,
 * is the one subtracted.  The act_atom records then hold theta* and the grid
 * winner's flat index.  0 (the default) keeps the grid-only search.
 * Changing the setting makes ragged plans built on this grid stale. */
ACT_API act_status act_set_refinement(act_grid *grid, int32_t steps);

/* Score and adjoint of continuous-parameter chirplets: for each channel b,
 * s_b = <r_b, g(theta_b)> with g the unit-norm real atom of Eq. (1), its
 * gradient ds_b/dtheta_b (tc, fc, logDt, c), and ds_b/dr_b = g(theta_b).
 *   theta      device, [channels][4] float64 (tc in samples, fc Hz, logDt,
 *              c Hz/s);
 *   residuals  device, [channels][n_samples] float32;
 *   score      device, [channels] float64 (the samples are FP32, the sums
 *              FP64: the score is not rounded to FP32 on output);
 *   grad_theta device, [channels][4] float64, may be NULL;
 *   atoms      device, [channels][n_samples] float32 (g(theta_b)), may be NULL.
 * n_samples 1..2048.  Enqueued on cuda_stream. */
ACT_API act_status act_chirplet_score(int32_t n_samples, double fs, const double *theta,
                                      const float *residuals, int32_t channels, double *score,
                                      double *grad_theta, float *atoms, void *cuda_stream);

/* Autotuner: times one search order of every candidate launch configuration
 * on this grid's dictionary with the caller's `channels` signals
 * [channels][n_samples] (device or host memory) as residuals, keeps the
 * fastest, and returns its time per order in *best_ms (may be NULL).
 * Candidates: resident CTAs per SM of the FP32 GEMV (1..4, as occupancy
 * allows), the bulk-copy streaming GEMV and, when the grid holds a BF16 dictionary,
 * tile width (128 or 256 atoms) x pipeline depth (2 .. what fits in shared
 * memory) of the tensor-core GEMM, each timed with its tile selection and
 * rescan; with an ACT_DICT_RECOMPUTE build, every valid (lags per thread,
 * warps, stages, CTAs per SM) combination of the template search instead
 * (act_set_shift_tuning).
 * Results never depend on the configuration, only the speed does.
 * Waits for the device.  Later act_decompose calls use the chosen
 * configuration. */
ACT_API act_status act_autotune(act_grid *grid, const float *signals, int32_t channels, void *cuda_stream,
                                double *best_ms);

/* The configuration in use: FP32 GEMV grid size in CTAs (-1: the
 * bulk-copy streaming GEMV, one CTA per SM), tensor-core tile width in atoms
 * and pipeline stages (0 and 0 without a BF16 dictionary). */
ACT_API act_status act_get_tuning(const act_grid *grid, int32_t *gemv_ctas, int32_t *bf16_tile_atoms,
                                  int32_t *bf16_stages);

/* Sets the configuration by hand: gemv_ctas > 0 sets the FP32 GEMV grid
 * (at most the resident limit), -1 selects the bulk-copy streaming GEMV (the
 * dictionary brought into shared memory by TMA bulk copies, one CTA per SM;
 * same scores and selections), 0 keeps the current choice;
 * bf16_tile_atoms (128 or 256) > 0 sets the
 * tensor-core tile width with bf16_stages pipeline stages (<= 0: the most
 * that fit).  Out-of-range values return ACT_ERR_INVALID_ARG. */
ACT_API act_status act_set_tuning(act_grid *grid, int32_t gemv_ctas, int32_t bf16_tile_atoms,
                                  int32_t bf16_stages);

/* Launch configuration of the template search (ACT_DICT_RECOMPUTE builds):
 * lags_per_thread (8, 16 or 32) time centres per thread, `warps` (1..8)
 * warps per CTA, whose product must divide the tc count rounded up to 32,
 * `stages` (1..3) shared-memory buffers of template chunks, and
 * ctas_per_sm persistent CTAs per SM (0: as many as fit).  act_autotune on
 * such a build times every valid combination and keeps the fastest.
 * Errors: ACT_ERR_NOT_BUILT without a template dictionary,
 * ACT_ERR_INVALID_ARG for an invalid combination.  Setting makes ragged
 * plans built on this grid stale. */
ACT_API act_status act_set_shift_tuning(act_grid *grid, int32_t lags_per_thread, int32_t warps, int32_t stages,
                                        int32_t ctas_per_sm);
ACT_API act_status act_get_shift_tuning(const act_grid *grid, int32_t *lags_per_thread, int32_t *warps,
                                        int32_t *stages, int32_t *ctas_per_sm);

/* Kernel-level measurement hooks used by the benchmark.
 * act_set_profiling(grid, 1) makes later act_decompose graphs record CUDA
 * events around every search of every order: before it, after its dominant
 * kernel (the FP32 GEMV, or the tensor-core GEMM) and after the whole search
 * (GEMM + tile selection + rescan + fallback).  act_profile_read waits for
 * the last act_decompose and returns, summed over its orders, the whole
 * search time (*search_ms) and the dominant kernel's time (*core_ms), the
 * number of orders timed, and in *kernels the number of kernels one
 * act_decompose launches. */
ACT_API act_status act_set_profiling(act_grid *grid, int32_t enable);
ACT_API act_status act_profile_read(act_grid *grid, double *search_ms, double *core_ms,
                                    int32_t *search_launches, int32_t *kernels);

/* Tensor-core search statistics since the grid was created (the dense BF16
 * search and the tensor-core template search): (channel, order) selections
 * resolved by the FP32 rescore of the flagged items, the total number of
 * items rescored for them (32-atom blocks of the dense search; (time centre,
 * 32-template block) items of the template search), and selections that took
 * the FP32 full search instead (more than 512 flagged blocks, or more than
 * 1,024 flagged items). */
ACT_API act_status act_bf16_stats(act_grid *grid, int64_t *resolved, int64_t *items_rescanned,
                                  int64_t *fallbacks);

/* Uneven batches (channels of different window lengths).
 *
 * act_ragged_plan_create prepares the decomposition of `channels` signals
 * laid end to end, channel c occupying samples offsets[c] .. offsets[c+1]-1
 * (offsets: host memory, [channels+1], offsets[0] = 0).  Each channel is
 * decomposed over the grid in grids[0 .. n_grids-1] whose n_samples equals
 * its length (one grid per length; every grid built on the same device).
 * Each length group uses its grid's search.  The whole batch -- gathers,
 * every group's n_atoms orders, scatters -- is captured once as one CUDA
 * graph whose length groups are independent branches.  The plan owns its
 * work buffers and search scratch (nothing a later call on a grid
 * reallocates); it shares each grid's dictionary and status word, so it must
 * be destroyed before the grids are.  Rebuilding a grid's dictionary or
 * changing its tuning, refinement, hierarchical settings or wait limit makes
 * the plan stale (act_ragged_decompose then returns ACT_ERR_NOT_BUILT).  Errors: ACT_ERR_INVALID_ARG (bad offsets, a length
 * with no grid, two grids of one length), ACT_ERR_NOT_BUILT, ACT_ERR_OOM. */
typedef struct act_ragged_plan act_ragged_plan;
ACT_API act_status act_ragged_plan_create(act_grid *const *grids, int32_t n_grids, const int64_t *offsets,
                                          int32_t channels, int32_t n_atoms, act_ragged_plan **out);

/* Runs the plan on signals (concatenated, [offsets[channels]] float32,
 * device or host).  Outputs as act_decompose, in the callers' channel order:
 * atoms_out and coeffs_out [channels][n_atoms], energy_out
 * [channels][n_atoms+1], residuals_out concatenated like the signals; any may
 * be NULL.  Waits only when a host buffer is involved. */
ACT_API act_status act_ragged_decompose(act_ragged_plan *plan, const float *signals, act_atom *atoms_out,
                                        float *coeffs_out, float *residuals_out, double *energy_out,
                                        void *cuda_stream);

/* Number of non-empty length groups, and kernels one act_ragged_decompose launches. */
ACT_API act_status act_ragged_plan_info(const act_ragged_plan *plan, int32_t *groups, int32_t *kernels);

ACT_API void act_ragged_plan_destroy(act_ragged_plan *plan);

/* act_search_noalloc -- the FP32 search (one projection + argmax step) for
 * callers that cannot allocate device memory.  The paper has no counterpart:
 * it exists because some callers may not call cudaMalloc -- a latency-bound
 * streaming loop that cannot take the device synchronisation an allocation
 * implies, or a process whose device memory is fully reserved by another
 * allocator.  It allocates nothing and uses no grid object.
 *
 * For each channel b it returns the atom i maximising |<D_i, r_b>| (lowest
 * index on ties) and that |score|, computed exactly as act_decompose's FP32
 * search computes them.
 *   dictionary  device, [n_atoms][row_stride] float32, caller-owned, rows
 *               zero beyond the window; 16-byte aligned;
 *   row_stride  128, 256, 384, 512, 1024 or 2048 floats;
 *   residuals   device, [channels][row_stride] float32, 16-byte aligned;
 *   channels    1 .. 256 (larger counts return ACT_ERR_UNSUPPORTED);
 *   best_index  device, [channels] int64 (-1 if a bounded device-side wait
 *               gave up or no finite score exists);
 *   best_score  device, [channels] float32 |score|.
 * Scratch: a fixed 2056-byte device array inside the library (one key per
 * channel plus a status word), held by every GPU that loads the library
 * until exit.  The first call on a device looks up that array's address with
 * cudaGetSymbolAddress while the device is current, and the first call with
 * each row stride, and with one and with several channels, loads that
 * kernel's code on the device.  Every call clears and reuses the same array,
 * so calls whose GPU work overlaps (different streams, or different host
 * threads on one device) race and must be serialised by the caller.
 * Enqueued on cuda_stream; nothing is waited for. */
ACT_API act_status act_search_noalloc(const float *dictionary, int64_t n_atoms, int32_t row_stride,
                                      const float *residuals, int32_t channels, int64_t *best_index,
                                      float *best_score, void *cuda_stream);

/* Frees the grid, its dictionary and all work buffers (waits for the device). */
ACT_API void act_destroy(act_grid *grid);

#ifdef __cplusplus
}
#endif

#endif /* ACT_H */
