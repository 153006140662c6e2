/*
 * hvox.h — C ABI of the GB300 HVOX transform library (libhvox.so).
 *
 * HVOX evaluates the radio-interferometric measurement sums of Sect. 2
 * (Eq. 2 and Eq. 3) with a 3-D type-3 non-uniform FFT (Sect. 3), chunked into
 * sub-problems (Eq. 8; Algorithms 1 and 2 of Sect. 3.2), each evaluated either by
 * the type-3 NUFFT (spread, FFT, interpolate, taper) or by direct summation when
 * that is cheaper (the small-block fallback of Sect. 3.1).
 *
 * Directions. With pixel unit vectors r_n, baselines p_k in wavelengths, weights
 * a_n (tessellation weights of Eq. 2; NULL means 1) and isign = +-1:
 *
 *   sky -> vis  (hvox_synthesize, alias hvox_dirty2vis):
 *        V_k = sum_n a_n I_n exp(+isign * j * 2 pi <p_k, r_n>)
 *   vis -> sky  (hvox_analyze, alias hvox_vis2dirty):
 *        I_n = a_n Re sum_k V_k exp(-isign * j * 2 pi <p_k, r_n>)
 *
 * isign = -1 reproduces Eq. 2 for sky -> vis. The paper calls the sky -> vis map
 * "analysis" and its adjoint "synthesis"; this library names sky -> vis
 * "synthesize" (synthesising visibilities from a sky model) and offers the unambiguous
 * aliases dirty2vis / vis2dirty, the names of the paper's user functions (Sect. 4). The
 * vis -> sky output is real (the paper's real=True adjoint, Listing 1): it is the
 * exact adjoint of sky -> vis under the real inner product.
 *
 * Accuracy: each output vector meets relative l2 error <= 10 * eps against the
 * exact sums (eps = 0 selects direct evaluation everywhere, Sect. 4), with the
 * upsampling the planner chooses (a caller-fixed upsampfac below 1.5 on FP32 grids has a
 * rounding floor of ~2^-24 (Phi(0)/Phi(pi/sigma))^2, 5e-4 at 1.25).
 *
 * Precision. HVOX_PREC_FP32: I is float[n_pix], V is interleaved complex
 * float[2 n_vis]. HVOX_PREC_FP64: double / double[2 n_vis]. AUTO picks FP32 for
 * eps >= 1e-6 and FP64 below. Coordinates, phases of large argument and plan-time
 * geometry are always FP64. FP64 plans evaluate direct sums in double-float
 * arithmetic on the FP32 units for eps >= 1e-9 (rounding ~3e-10) and with FP64
 * kernels below 1e-9 (~100x slower, so the planner gives such plans more NUFFT
 * work); their NUFFT sub-problems run on FP64 grids. Tolerances that would need a
 * kernel wider than 16 cells at every upsampling (eps below ~1e-14) return
 * HVOX_EUNSUPPORTED.
 *
 * Memory. Coordinates and weights passed to hvox_plan may be host or device
 * pointers; they are copied (and permuted to chunk order) into plan-owned device
 * memory, so the caller may free them on return. I and V passed to the transform
 * calls may be device pointers (the fast path) or host pointers (then the call
 * copies through plan-owned staging buffers and synchronises its stream before
 * returning). Outputs are overwritten, never accumulated into.
 *
 * Streams and errors. Work is enqueued on opts.stream (NULL = the legacy default
 * stream). Device pointers make the transform calls asynchronous: a device-side
 * failure is reported by the next call on the plan or by hvox_sync. Argument
 * errors return HVOX_EINVAL before any work is enqueued. A failed hvox_plan
 * frees everything it allocated. A plan must not be used from two host threads at
 * once; different plans may run concurrently on different streams.
 * hvox_last_error() returns a thread-local message for the last failure.
 */
#ifndef HVOX_H
#define HVOX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hvox_plan_s *hvox_plan_t;

typedef enum {
    HVOX_OK = 0,
    HVOX_EINVAL = 1,        /* bad argument; nothing was enqueued */
    HVOX_ENOMEM = 2,        /* device or host allocation failed */
    HVOX_ECUDA = 3,         /* a CUDA runtime or cuFFT call failed */
    HVOX_ETIMEOUT = 4,      /* reserved: no kernel of this library waits on a flag, a peer
                               or another kernel, so no call returns it */
    HVOX_EUNSUPPORTED = 5,  /* option combination not supported */
    HVOX_EINTERNAL = 6      /* internal invariant violated; also the plan's device error
                               word: a kernel found a spreading or interpolation window
                               outside its grid, clamped it (no out-of-bounds access) and
                               set the word, which hvox_sync, hvox_get_stats and the calls
                               that synchronise (host pointers) report and clear */
} hvox_status;

typedef enum { HVOX_PREC_AUTO = 0, HVOX_PREC_FP32 = 1, HVOX_PREC_FP64 = 2 } hvox_prec;

typedef enum {
    HVOX_MODE_AUTO = 0,     /* per-block choice NUFFT vs direct by the cost model */
    HVOX_MODE_NUFFT = 1,    /* every block by type-3 NUFFT */
    HVOX_MODE_DIRECT = 2    /* every block by direct summation (the eps = 0 semantics) */
} hvox_mode;

/* Options. A zero-initialised struct selects the defaults. */
typedef struct {
    int32_t precision;           /* hvox_prec */
    int32_t mode;                /* hvox_mode */
    double upsampfac;            /* sigma of both NUFFT stages, in [1.25, 4]; 0 -> chosen by
                                    the planner among 2, 1.5 and 1.25 */
    double chunk_budget_bytes;   /* FFT-grid budget B of one sub-problem (Algorithm 1);
                                    0 -> chosen by the planner's cost model. A fixed budget
                                    also caps the grid bytes of a wave (the sub-problems run
                                    together; otherwise up to 16 GiB). A budget that
                                    cannot hold a grid of 2w cells per dimension, or that
                                    would cut the job into more than 2^24 candidate
                                    sub-problems, makes hvox_plan fail with HVOX_EINVAL */
    double anisotropy;           /* Algorithm 1 alpha >= 1; 0 -> 1 (isotropic optimum) */
    double direct_threshold;     /* < 0 or 0 -> cost model; > 0: a block with
                                    n_pix_blk * n_vis_blk <= threshold is direct */
    double search_threshold;     /* seconds; a job whose direct evaluation (both directions)
                                    is modelled below this is planned as direct sums
                                    without searching partitions. 0 -> 0.01 s. Callers
                                    that use a plan once (per-request serving) pass more,
                                    since the search costs ~1-3 us per point. */
    int32_t ntrans;              /* number of stacked inputs on one geometry; 0 -> 1 */
    int32_t plain;               /* 1: the plain reference form: FP64 arithmetic in every
                                    kernel, blocks launched one by one (eager launches on
                                    the same lanes, no graph) */
    int32_t graphs;              /* CUDA graphs: 0 -> for plans with NUFFT sub-problems;
                                    1 -> for every plan; -1 -> never (eager launches).
                                    The first call of each direction runs eagerly; the
                                    second captures the work between the permutations
                                    (zeroing, direct launch, every sub-problem on its lane)
                                    into one graph, which later calls replay. Ignored by
                                    the plain form. */
    int32_t chunk_order;         /* 1: the caller passes and receives I and V in the plan's
                                    chunk order (hvox_plan_order gives it), so the
                                    permutations are skipped; the weights a_n are still
                                    applied. 0: the caller's own point order. */
    void *stream;                /* cudaStream_t; NULL = legacy default stream */
    int32_t factor;              /* which set's spreading is shared across sub-problems (the
                                    factored evaluation of Sect. 3, Table 1's "theory" row):
                                    0 -> chosen by the cost model among the box splits it
                                    searches, which include both factored forms;
                                    1 -> pixels: one baseline box spans every baseline, so
                                    each pixel is spread (and gathered) once and the pixel
                                    chunks shrink to keep Algorithm 1's grid size;
                                    2 -> baselines: one pixel box spans the sky, so each
                                    baseline is spread (and gathered) once.
                                    A shared spread must resolve every frequency its
                                    sub-problems read (the kernel transform is evaluated at
                                    the full p, not p - D_j), so sharing is exact only with
                                    a box that spans the other set. */
    int32_t autotune;            /* 1: measure at plan time (a few extra launches and a
                                    probe during hvox_plan): (a) the kernel width: the
                                    NUFFT sub-problem with the most points (its pixels and
                                    up to 2,048 of its baselines) is evaluated by direct
                                    sums and by the NUFFT with 1 and 2 cells less than the
                                    width rule gives; the narrowest width whose measured
                                    relative l2 error is within 2.5 eps is kept and the job
                                    re-planned with it (hvox_info.probe_error); (b) which
                                    bin size (points per spreading CTA: 32, 64 or 128)
                                    spreads fastest, per direction. 0: the width rule and
                                    bins of 128 */
    int32_t kernel_width;        /* 0: the width rule; 2..16: this width for every upsampling
                                    (shape parameter from the same rule); HVOX_EINVAL else */
} hvox_opts;

/* Plan summary (filled by hvox_plan_info). */
typedef struct {
    int64_t n_pix, n_vis;
    int32_t precision;           /* resolved hvox_prec */
    int32_t isign;
    double eps;
    int32_t w;                   /* ES kernel width (grid cells per dimension) */
    double beta;                 /* ES kernel shape parameter */
    double upsampfac;
    double budget_bytes;         /* B used by Algorithm 1 */
    double t;                    /* Algorithm 1 scale: h = t B_k, eta = t P_k */
    double h[3], eta[3];         /* maximal Heisenberg dimensions (wavelengths / unit) */
    int64_t n_pix_chunks, n_vis_chunks;
    int64_t n_nufft_blocks;      /* sub-problems evaluated by type-3 NUFFT */
    int64_t n_direct_rects;      /* rectangles of direct work after merging */
    double direct_pairs;         /* sum of n_pix * n_vis over direct sub-problems */
    double nufft_points;         /* sum of n_pix + n_vis over NUFFT sub-problems */
    double nufft_cells;          /* sum of FFT-grid cells over NUFFT sub-problems */
    double max_grid_bytes;       /* largest sub-problem grid (spread + FFT grids) */
    double workspace_bytes;      /* plan-owned device memory */
    double plan_seconds;         /* wall time of hvox_plan */
    double model_seconds;        /* cost-model estimate of one sky->vis plus one vis->sky */
    int32_t graph_state;         /* 0: eager launches so far; 1: a graph has been captured
                                    and is replayed; -1: capture failed, eager launches */
    /* Work of one sky->vis (the same again for vis->sky) summed over NUFFT sub-problems,
       the quantities the cost model charges: */
    double nufft_pix_points;     /* pixels spread (and, in vis->sky, gathered) */
    double nufft_vis_points;     /* baselines gathered (and, in vis->sky, spread) */
    double spread_cells;         /* n1 grid cells (M1) */
    double fft_work;             /* M2 log2 M2 over the FFT grids */
    double box_ratio;            /* pixel box dims = ratio x Algorithm 1's, baseline box dims
                                    = Algorithm 1's / ratio (1: the isotropic optimum) */
    int32_t spread_bin_pix;      /* points per spreading CTA, pixels (sky -> vis) */
    int32_t spread_bin_vis;      /* points per spreading CTA, baselines (vis -> sky) */
    int32_t kernel_width_rule;   /* the width rule's kernel width at the plan's upsampling */
    double probe_error;          /* autotune: measured error of the chosen width on the probe
                                    sub-problem; -1 when not measured */
    int32_t fft_batches;         /* batched FFTs of a transform (one per grid shape and wave) */
    int32_t fft_batches_df;      /* of those, FP64 grids transformed in double-float arithmetic
                                    on the FP32 pipes (the rest: cuFFT) */
    int32_t direct_vpt;          /* owners (points) per thread of the direct kernels, 2 or 4 */
} hvox_info;

/*
 * hvox_plan — build a plan: Algorithm 1 (box dimensions), Algorithm 2 (chunking of
 * pixels and baselines), the NUFFT-or-direct choice per sub-problem (Sect. 3.1),
 * the chunk-order permutation (Sect. 4), grid sizes and kernel tables.
 *   pix_xyz    (n_pix, 3) row-major FP64 pixel positions (unit vectors; any finite
 *              positions are accepted). Host or device pointer.
 *   uvw        (n_vis, 3) row-major FP64 baselines in wavelengths. Host or device.
 *   pix_weight (n_pix) FP64 weights a_n, or NULL for 1. Host or device.
 *   eps        target relative l2 error; 0 selects direct evaluation everywhere.
 *   isign      +1 or -1 (sign of the exponent of sky -> vis).
 *   opts       may be NULL (defaults).
 *   out        receives the plan handle; set to NULL on failure.
 * Errors: HVOX_EINVAL for n_pix < 1, n_vis < 1, NULL pointers, eps < 0 or not finite,
 * |isign| != 1, non-finite coordinates, bad options (an infeasible chunk budget);
 * HVOX_EUNSUPPORTED for a tolerance no 16-cell kernel reaches; HVOX_ENOMEM; HVOX_ECUDA.
 */
hvox_status hvox_plan(const double *pix_xyz, int64_t n_pix, const double *uvw, int64_t n_vis,
                      const double *pix_weight, double eps, int isign, const hvox_opts *opts,
                      hvox_plan_t *out);

/* sky -> vis. I: ntrans * n_pix reals, V: ntrans * n_vis complex (interleaved), in the
 * plan precision; transform t occupies I[t n_pix ...], V[2 t n_vis ...]. */
hvox_status hvox_synthesize(hvox_plan_t plan, const void *I, void *V);

/* vis -> sky (exact adjoint of hvox_synthesize, real part). Layouts as above. */
hvox_status hvox_analyze(hvox_plan_t plan, const void *V, void *I);

/* Free every resource of the plan (waits for its stream). NULL is accepted. */
hvox_status hvox_destroy(hvox_plan_t plan);

/* Complex sky (the paper's real=False form of Listing 1): I is ntrans = 1 complex
 * array of n_pix (float2/double2 interleaved in the plan's precision), V as above; both
 * device pointers (HVOX_EINVAL for host pointers, HVOX_EUNSUPPORTED for ntrans > 1).
 *   hvox_synthesize_complex: V_k = sum_n a_n I_n exp(+isign j 2 pi <p_k, r_n>)
 *   hvox_analyze_complex:    I_n = a_n sum_k V_k exp(-isign j 2 pi <p_k, r_n>) (no real part)
 * Each runs the real transform twice (linearity: A (x + j y) = A x + j A y, and
 * A^H v = Re(A^H v) + j Re(A^H (-j v))). */
hvox_status hvox_synthesize_complex(hvox_plan_t plan, const void *I, void *V);
hvox_status hvox_analyze_complex(hvox_plan_t plan, const void *V, void *I);

/*
 * hvox_synthesize_batch / hvox_analyze_batch — the transforms of n distinct plans in one
 * call, the parallel sub-transforms of Sect. 3 carried across jobs: on `stream`, each
 * plan's input permutation and NUFFT sub-problems as in hvox_synthesize / hvox_analyze,
 * but the direct sub-problems of every plan whose direct sums run on the FP32 or the
 * double-float kernels merged into one launch per kernel form (their work items in one
 * list, largest first, each tagged with its plan), so that small jobs share kernels and
 * their dynamic schedule. Plans with FP64 direct sums (the plain form, eps < 1e-9) launch
 * theirs separately.
 *   plans      n distinct plans on one device, each with ntrans = 1.
 *   I / V      n device pointers each (plan i's input and output, layouts as above).
 *   stream     cudaStream_t or NULL (legacy default stream). The call is ordered after
 *              the work already queued on every plan's own stream, and each plan's stream
 *              is ordered after the call; the call returns once everything is enqueued.
 *   direct_launches  may be NULL; receives the number of direct-sum launches made.
 * Profiling (hvox_profile) covers the plans' NUFFT stages; merged direct launches are
 * not bracketed. Errors: HVOX_EINVAL for NULL or host pointers, a repeated plan or
 * plans on different devices, n < 0; HVOX_EUNSUPPORTED for ntrans > 1; HVOX_ECUDA.
 * n = 0 does nothing.
 */
hvox_status hvox_synthesize_batch(const hvox_plan_t *plans, const void *const *I, void *const *V, int32_t n,
                                  void *stream, int32_t *direct_launches);
hvox_status hvox_analyze_batch(const hvox_plan_t *plans, const void *const *V, void *const *I, int32_t n,
                               void *stream, int32_t *direct_launches);

/* Aliases with the direction in the name. */
hvox_status hvox_dirty2vis(hvox_plan_t plan, const void *I, void *V);
hvox_status hvox_vis2dirty(hvox_plan_t plan, const void *V, void *I);

/* Plan summary. */
hvox_status hvox_plan_info(hvox_plan_t plan, hvox_info *info);

/* Chunk labels chosen by the plan, in the caller's original point order:
 * pix_chunk[n] (n_pix entries) and vis_chunk[k] (n_vis entries), host pointers,
 * either may be NULL. Chunks are numbered as Algorithm 2 creates them. */
hvox_status hvox_plan_chunks(hvox_plan_t plan, int64_t *pix_chunk, int64_t *vis_chunk);

/* The plan's chunk order (Sect. 4: inputs reordered so that every sub-problem reads
 * contiguous slices): pix_order[m] (n_pix entries) is the caller's index of the pixel at
 * chunk position m, vis_order[m] (n_vis entries) likewise for baselines. Host pointers,
 * either may be NULL. A caller that keeps its data in this order plans with
 * hvox_opts.chunk_order = 1. */
hvox_status hvox_plan_order(hvox_plan_t plan, int64_t *pix_order, int64_t *vis_order);

/* Stages of a transform, for hvox_get_stats. */
enum {
    HVOX_STAGE_PERMUTE = 0,  /* caller order <-> chunk order, weights (Sect. 4) */
    HVOX_STAGE_DIRECT = 1,   /* direct sub-problems (Sect. 3.1 fallback) */
    HVOX_STAGE_SPREAD = 2,   /* NUFFT spreading (step 1 of the type-3 transform) */
    HVOX_STAGE_DECONV = 3,   /* deconvolve + zero-pad / crop (taper of step 1) */
    HVOX_STAGE_FFT = 4,      /* uniform 3-D FFT (cuFFT, step 2) */
    HVOX_STAGE_INTERP = 5,   /* NUFFT interpolation with taper (steps 3-4) */
    HVOX_STAGE_ZERO = 6,     /* clearing accumulators and grids */
    HVOX_NUM_STAGES = 8
};

typedef struct {
    double ms[HVOX_NUM_STAGES];        /* device time per stage: CUDA events recorded around
                                          each stage on the stream that runs it (0 unless
                                          profiling). Stages of sub-problems on concurrent lanes
                                          overlap one another and the direct sums, so with more
                                          than one lane the times need not add up to the step */
    int64_t launches[HVOX_NUM_STAGES]; /* kernel launches of this library per stage (FFT: cuFFT
                                          executions; ZERO: memsets) */
    int64_t transforms;                /* transforms run since the last reset */
} hvox_stats;

/* Reset the statistics and turn event timing on (enable = 1 or 2) or off (0). Launch
 * counts are always collected. enable = 1 times the transforms as they normally run
 * (sub-problems on concurrent lanes, CUDA graphs), so a stage's time also counts the time
 * its kernels wait for SMs held by concurrent work. enable = 2 is the serial form for
 * per-kernel measurement: every stage runs alone on the plan's stream, without lanes or
 * graphs, so each stage time is the device time of its own launches (the transforms run
 * slower meanwhile). HVOX_EINVAL for other values. */
hvox_status hvox_profile(hvox_plan_t plan, int enable);

/* Statistics since the last hvox_profile call (waits for the plan's stream). */
hvox_status hvox_get_stats(hvox_plan_t plan, hvox_stats *out);

/* Wait for the plan's stream and report any device-side error: a CUDA error, or the
 * plan's device error word (HVOX_EINTERNAL; the word is cleared by the report). */
hvox_status hvox_sync(hvox_plan_t plan);

/* Host-only dry run of hvox_plan: the partition, the per-sub-problem choices and the
 * cost-model estimate, without touching a GPU (host pointers only). Fills the plan
 * fields of *info (workspace_bytes is an estimate; plan_seconds is the planning time). */
hvox_status hvox_plan_dry(const double *pix_xyz, int64_t n_pix, const double *uvw, int64_t n_vis, double eps,
                          const hvox_opts *opts, hvox_info *info);

/* Upper bound of the device memory a plan with these sizes and options could own
 * (admission control): coordinates, permutations, call buffers and, unless the job is
 * planned as direct sums without a search, up to four lanes of grids and cuFFT work
 * areas within the chunk budget (8 GiB when the planner chooses). 0 on error. */
double hvox_estimate_bytes(int64_t n_pix, int64_t n_vis, double eps, const hvox_opts *opts);

/* Thread-local message describing the last failure ("" if none). */
const char *hvox_last_error(void);

/* Library version string. */
const char *hvox_version(void);

/* ---------------------------------------------------------------------------
 * Direct sky -> vis evaluation that allocates nothing (no counterpart in the paper).
 *
 * For callers that cannot call cudaMalloc: code running inside another framework that has
 * reserved the device's memory for its own pool, and per-iteration loops (for example a
 * calibration solver predicting visibilities from a sky model every step) where an
 * allocation, and the device synchronisation that freeing brings, is not allowed.
 *
 * Computes V_k = sum_n I_n exp(+isign j 2 pi <p_k, r_n>) by direct summation in FP32
 * (phase fractions from exact hi/lo products, as in the planned FP32 path; relative l2
 * error ~1e-6), without weights, in the caller's point order.
 *   pix_xyz (n_pix, 3) FP64, uvw (n_vis, 3) FP64 wavelengths, I float[n_pix],
 *   V interleaved complex float[2 n_vis] (overwritten): all DEVICE pointers (host
 *   pointers are rejected with HVOX_EINVAL). stream: cudaStream_t or NULL.
 * Limit: n_pix + n_vis <= 524,288 (HVOX_EINVAL beyond, nothing enqueued). The working
 * memory is one static device array of 16 MiB (coordinate splits), held on every GPU
 * that loads it until the process exits; the call itself calls no cudaMalloc, cudaFree
 * or allocating library routine. CUDA loads device code lazily by default, so the array
 * is reserved on a device by the first call of this function there (or the first
 * direct-sum launch of any plan there): a caller whose framework will take the whole
 * device memory pool should make one call before the pool fills, else that first call
 * can fail with HVOX_ECUDA (out of memory). The first call on a device also looks up the
 * array's device address (cudaGetSymbolAddress) with the device current; make that first
 * call before any stream capture. All calls share the array and it keeps the last call's
 * contents, so calls whose work overlaps on the GPU (different streams, or different
 * host threads) race: serialise them. The sum over pixels runs in segments of 4096
 * pixels whose partial sums meet through atomic adds, so the last bits of V may differ
 * between calls. Asynchronous on `stream`.
 */
hvox_status hvox_direct_synthesize_noalloc(const double *pix_xyz, int64_t n_pix, const double *uvw, int64_t n_vis,
                                           const float *I, float *V, int isign, void *stream);

/* ---------------------------------------------------------------------------
 * Host-only planning primitives (no GPU needed), exposed for testing and for
 * callers that want to inspect a partition before planning.
 * --------------------------------------------------------------------------- */

/* ES kernel parameters for tolerance eps and upsampling sigma (Barnett, Magland and
 * af Klinteberg 2019, the type-3 engine the paper uses): width w = ceil(ln(1/eps) /
 * (pi sqrt(1 - 1/sigma))) grid cells and beta = 0.97 pi w (1 - 1/(2 sigma)). */
hvox_status hvox_es_params(double eps, double sigma, int32_t *w, double *beta);

/* Fourier transform of the ES kernel phi(z) = exp(beta (sqrt(1 - (2z/w)^2) - 1)),
 * |z| <= w/2 (grid units): out[i] = int phi(z) cos(xi[i] z) dz, by Gauss-Legendre
 * quadrature (the deconvolution factors of the spread and interpolation steps). */
hvox_status hvox_es_ft(int32_t w, double beta, const double *xi, int64_t n, double *out);

/* Algorithm 1: largest t in (0, 1] such that the padded grids of a sub-problem with
 * extents eta = t P (pixels) and h = t B (wavelengths) fit budget_bytes, for
 * upsampling sigma, kernel width w and complex element size elem_bytes. */
hvox_status hvox_box_dims(const double P[3], const double B[3], double budget_bytes, double sigma,
                          int32_t w, int32_t elem_bytes, double eta[3], double h[3], double *t);

/* The planner's cost model (the GPU counterpart of the paper's regression of stage runtimes,
 * Sect. 4 and its appendix): seconds per unit of work for plans of this precision
 * (HVOX_PREC_FP32 or HVOX_PREC_FP64) and form (plain = 1: FP64 kernels). rates[0..7] =
 * direct pair (one direction), spreading tap through a shared tile, spreading tap straight
 * into the grid, interpolation tap, FFT cell per log2(cells), grid-pass cell, fixed seconds
 * per sub-problem and direction, and the shared tile's capacity in cells. */
hvox_status hvox_cost_model(int32_t precision, int32_t plain, double rates[8]);

/* Algorithm 2: chunk labels of n points (row-major (n, 3), host pointer) for maximal
 * box dimensions h; labels[n] host output, *n_chunks the chunk count. */
hvox_status hvox_chunk_points(const double *xyz, int64_t n, const double h[3], int64_t *labels,
                              int64_t *n_chunks);

#ifdef __cplusplus
}
#endif

#endif /* HVOX_H */
