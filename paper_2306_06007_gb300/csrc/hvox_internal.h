// Internal declarations shared by the host planner/executor and the CUDA kernels.
#pragma once

#include <cuda_runtime.h>
#include <cufft.h>

#include <cstdint>
#include <map>
#include <memory>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/hvox.h"

namespace hvox {

// ------------------------------------------------------------------ errors

void set_error(const std::string &msg);
const char *get_error();

struct Error {
    hvox_status code;
    std::string msg;
};

// Throwing helpers used inside the library; the ABI layer converts to codes.
[[noreturn]] void fail(hvox_status code, const std::string &msg);
void check_cuda(cudaError_t e, const char *what);
void check_cufft(cufftResult r, const char *what);

// Host-side fault injection for tests. HVOX_FAULT = "site:n[,site:n...]" makes the n-th
// event of each named site (counted from the moment the variable last changed) fail the
// way the real failure would:
//   alloc    a device allocation (HVOX_ENOMEM, everything allocated so far freed);
//   cufft    a cuFFT plan creation (HVOX_ECUDA);
//   capture  a CUDA-graph capture (the plan falls back to eager launches);
//   window   the pixel scale of the NUFFT sub-problem with the most pixels is multiplied
//            by 4 on the host, so its kernels clamp the pixels' windows into the grid and
//            set the device error word (hvox_sync then returns HVOX_EINTERNAL).
// No GPU fault is involved: every injected failure is raised or prepared on the host.
bool fault_hit(const char *site);

// Bits of a plan's device error word, set by kernels that had to clamp an index.
enum : int {
    kDevErrPixWindow = 1,   // a pixel window outside the n1 grid (clamped into it)
    kDevErrVisWindow = 2    // a baseline window beyond one period of the n2 grid (clamped)
};

// ------------------------------------------------------------------ ES kernel

struct ESKernel {
    int w = 0;          // width in grid cells per dimension
    double beta = 0.0;  // shape
};

ESKernel es_params(double eps, double sigma);
int es_width(double eps, double sigma);  // the width rule of es_params, without its limit of 16
ESKernel es_with_width(int w, double sigma);  // a caller-fixed width, the same shape rule
// The kernel for the tightened tolerance eps_tight, or the 16-cell kernel when that one
// would be wider and eps itself fits in 16 cells (a caller-fixed upsampling).
ESKernel es_params_within(double eps_tight, double eps, double sigma);
// Gauss-Legendre nodes/weights on [-1, 1].
void gauss_legendre(int q, std::vector<double> &x, std::vector<double> &wt);
// int phi(z) cos(xi z) dz over |z| <= w/2 for each xi (host FP64).
void es_ft(const ESKernel &k, const double *xi, int64_t n, double *out);
int es_quad_nodes(const ESKernel &k);
void es_ft_nodes(const ESKernel &k, std::vector<double> &z, std::vector<double> &f);
void fit_inv_phi(const ESKernel &k, double tau_max, double tol, std::vector<double> &coef);

// ------------------------------------------------------------------ planning

int64_t smooth_even(int64_t n);
void grid_sizes(double extent_pix, double extent_vis, double sigma, int w, int64_t &n1, int64_t &n2);
double grid_bytes(const double P[3], const double B[3], double sigma, int w, int elem_bytes);
double box_dims(const double P[3], const double B[3], double budget, double sigma, int w, int elem_bytes,
                double eta[3], double h[3]);
// Algorithm 2. labels[i] in [0, n_chunks).
int64_t chunk_points(const double *xyz, int64_t n, const double h[3], std::vector<int64_t> &labels);

// One sub-problem evaluated by type-3 NUFFT.
struct NufftBlock {
    int64_t pix_chunk = 0, vis_chunk = 0;
    int64_t p0 = 0, p1 = 0;   // pixel range in chunk order
    int64_t v0 = 0, v1 = 0;   // baseline range in chunk order
    double C[3] = {0, 0, 0};  // pixel-box centre
    double D[3] = {0, 0, 0};  // baseline-box centre (wavelengths)
    double a[3] = {0, 0, 0};  // spread-grid cells per unit of r
    int64_t n1[3] = {0, 0, 0};
    int64_t n2[3] = {0, 0, 0};
    int64_t psi_off = 0;      // offset of this block's 1/psi tables (n1[0]+n1[1]+n1[2])
    double cost = 0.0;
};

// A rectangle of direct work: pixels [p0, p1) x baselines [v0, v1) (chunk order).
struct DirectRect {
    int64_t p0, p1, v0, v1;
};

// Work item of the direct kernels: owner tile [o0, o1) and streamed range [s0, s1).
struct WorkItem {
    int32_t o0, o1, s0, s1;
};

// Device pointers of one job of a direct launch (one plan's chunk-ordered buffers): owner
// coordinates (sky -> vis: baselines, vis -> sky: pixels) and streamed coordinates as
// hi / lo float4 splits, the streamed values (c or V), the owners' accumulators, and the
// exponent's sign.
struct DirectJob {
    const float4 *own_hi, *own_lo, *str_hi, *str_lo;
    const void *val;
    void *acc;
    float sgn;
};

struct CostModel {
    double direct_pair = 0;      // seconds per (pixel, baseline) pair, one direction
    double scatter_smem = 0;     // seconds per tap of spreading through a shared-memory tile
    double scatter_global = 0;   // seconds per tap of spreading straight into the grid
    double gather_tap = 0;       // seconds per tap of interpolation
    double fft_cell = 0;         // seconds per FFT-grid cell per log2(cells)
    double grid_cell = 0;        // seconds per grid cell of pad/crop/zero passes
    double block_fixed = 0;      // seconds of fixed overhead per NUFFT block and direction
    double tile_cells = 0;       // shared-memory tile capacity of the spreading kernels
};

// z2z_fft: FP64 grids go through cuFFT Z2Z instead of the double-float FFT.
CostModel default_cost_model(int prec, bool plain, int w, bool z2z_fft = false);

struct PartitionResult {
    double t = 1.0, h[3] = {0, 0, 0}, eta[3] = {0, 0, 0}, budget = 0;
    double sigma = 2.0;       // upsampling chosen for the NUFFT sub-problems
    ESKernel es;              // kernel for that upsampling
    std::vector<int64_t> pix_label, vis_label;  // original index -> chunk label
    int64_t n_pix_chunks = 0, n_vis_chunks = 0;
    std::vector<int64_t> pix_perm, vis_perm;    // chunk-order position -> original index
    std::vector<int64_t> pix_chunk_start, vis_chunk_start;  // per ordered chunk, size chunks+1
    std::vector<int64_t> pix_chunk_label, vis_chunk_label;  // ordered chunk -> Algorithm 2 label
    std::vector<NufftBlock> blocks;
    std::vector<DirectRect> rects;
    double direct_pairs = 0, nufft_points = 0, nufft_cells = 0, max_grid_bytes = 0;
    double nufft_pix_points = 0, nufft_vis_points = 0, spread_cells = 0, fft_work = 0;
    double box_ratio = 1.0;   // eta / h split relative to Algorithm 1's isotropic boxes
    double model_seconds = 0;
};

struct PlanInputs {
    const double *pix;     // host (n_pix, 3)
    const double *uvw;     // host (n_vis, 3)
    int64_t n_pix, n_vis;
    double sigma;          // upsampling (used when sigma_auto is false)
    ESKernel es;
    bool sigma_auto = false;  // choose sigma in {2, 1.5, 1.25} by the cost model
    double eps_es = 1e-6;     // tolerance given to the kernel-width rule
    int prec;              // 1 fp32, 2 fp64
    int mode;
    bool plain;
    bool direct_f64 = false;  // direct sums by the FP64 kernels (plain form, eps < 1e-9)
    double budget;         // 0 -> search
    double max_budget = 0; // > 0: largest budget the search may pick (device memory)
    double direct_threshold;
    double search_threshold = 0.01;  // seconds of modelled direct work below which no search
    int elem_bytes;
    int factor = 0;        // hvox_opts.factor: 0 searched, 1 one baseline box, 2 one pixel box
    int fixed_w = 0;       // > 0: kernel width for every upsampling (shape from the width rule)
    bool z2z_fft = false;  // FP64 grids by cuFFT Z2Z (cost model), see dfft_wanted
};

PartitionResult make_partition(const PlanInputs &in);

// ------------------------------------------------------------------ device buffers

struct DevBuf {
    void *ptr = nullptr;
    size_t bytes = 0;
    void alloc(size_t n);
    void free_();
    ~DevBuf() { free_(); }
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    template <typename T> T *as() const { return reinterpret_cast<T *>(ptr); }
};

// Device-side description of a NUFFT block: FP64 geometry and its float hi/lo splits
// (passed by value to the kernels).
struct NufftDev {
    int64_t p0, np, v0, nv;
    int32_t n1[3], n2[3];
    double C[3], D[3], a[3];
    double n2a[3];    // n2 / a (0 when a = 0)
    double tpa64[3];  // 2 pi / a (0 when a = 0)
    float Ch[3], Cl[3], Dh[3], Dl[3], ah[3], al[3], n2ah[3], n2al[3], tpa[3];
    int64_t psi_off;
    int *err;         // the plan's device error word (kDevErr* bits)
    int64_t g1_off;   // its spread grid: n1 cells (x fastest) from cell g1_off of its lane's g1
    int64_t g2_off;   // its FFT grid: cell (x, y, z) at g2_off + z * zs2 + y * n2[0] + x of g2
    int64_t zs2;      // z-plane stride of the FFT grid in cells (a batch interleaves its planes)
};

template <typename T> struct CplxOf;
template <> struct CplxOf<float> { using type = float2; };
template <> struct CplxOf<double> { using type = double2; };

// cuFFT plans of one FFT-grid shape and batch. Pruned form (xy and z set): the 3-D
// transform as 2-D transforms of the n1 band's z planes (two slabs of n1z/2 planes, at the
// start and the end of the grid) and 1-D transforms along z of every column; the other z
// planes hold only zeros before the transform (sky -> vis) or are not read after it (vis ->
// sky), so their 2-D transforms are skipped. Full form (full set): one 3-D plan per grid.
struct FftPlans {
    cufftHandle full = 0, xy = 0, z = 0;
};

// One length of the double-float FFT (k_dffft.cu): radices of its Stockham stages, the
// divisor of each stage's butterfly index as a multiplier (floor(2^32 / Ns) + 1, exact for
// indices below 2^14 and Ns >= 2), the odd radices' DFT coefficients cos and sin of
// 2 pi m / r (m = q k mod r; r = 3 at [0], 5 at [1, 5), 7 at [5, 14), entry (q - 1) h + k - 1
// with h = r / 2) and the twiddle table exp(2 pi i q / n), q < n; every value a float pair
// (cos h, cos l, sin h, sin l).
constexpr int kDfftMaxStages = 16;
struct DfftDev {
    int n = 0, stages = 0;
    int radix[kDfftMaxStages] = {0};
    unsigned ns_magic[kDfftMaxStages] = {0};
    float4 odd[14];
    const float4 *tw = nullptr;
};

// The batched transforms of K sub-problems of one grid shape inside a wave: their FFT
// grids interleave z planes (plane z of grid g at g2 + (z K + g) * n2x n2y), so that each
// band slab of all K grids is one contiguous run of planes (one batched 2-D call) and
// every column of every grid is one strided 1-D transform along z (one batched call).
struct FftBatch {
    void *g2 = nullptr;       // plane 0 of grid 0
    int64_t n2[3] = {0, 0, 0};
    int64_t half = 0;         // n1z / 2
    int64_t K = 1;
    FftPlans plans;
    bool df = false;          // FP64 grids through the double-float FFT instead of cuFFT Z2Z
                              // (FP64 cells in, double-float cells out: Plan::df_grids)
    DfftDev dx, dy, dz;       // its three lengths
    int64_t h1y = 0;          // n1y / 2: the band rows are [0, h1y) and [n2y - h1y, n2y)
};

// Double-float FFT (k_dffft.cu): radices of length n (false when a factor other than 2, 3,
// 5, 7 remains), whether a grid shape is covered, the twiddle table of a length, and the
// batched pruned 3-D transform of one batch (sign -1 or +1; band_input as fft_batch).
bool dfft_factor(int n, DfftDev &d);
bool dfft_supported(const int64_t n2[3]);
void dfft_twiddles(int n, std::vector<float> &tab);
int dfft_batch(const FftBatch &f, int sign, bool band_input, cudaStream_t s);

// A wave: sub-problems [b0, b0 + nb) of the plan's descriptor array, run together: one
// clearing, spreading, deconvolution and interpolation launch each (a 2-D launch grid over
// (tile, sub-problem)) and one batched FFT set per grid shape. Its grids live in the
// buffers of its lane (n1 grids back to back, then the n2 grids).
struct Wave {
    int b0 = 0, nb = 0;
    int lane = 0;
    int64_t g1_cells = 0, g2_cells = 0;      // grid cells of the wave (each set contiguous)
    int64_t max_np = 0, max_nv = 0;          // most pixels / baselines of one sub-problem
    int64_t max_rows1 = 0, max_rows2 = 0;    // most n1 rows (n1y n1z) / n2 rows (n2y n2z)
    std::vector<FftBatch> ffts;
    double cost = 0.0;
};

// Plan-wide arguments of the NUFFT launchers.
template <typename T> struct NufftArgs {
    int w = 0;
    double beta = 0.0;
    int isign = -1;
    const NufftDev *descs = nullptr;  // device array of the plan's sub-problem descriptors
    const T *ipsi = nullptr;
    const float4 *pix_hi = nullptr, *pix_lo = nullptr, *vis_hi = nullptr, *vis_lo = nullptr;
    const double *pix_soa = nullptr, *vis_soa = nullptr;
    int64_t n_pix = 0, n_vis = 0;
    const T *cheb = nullptr;   // Chebyshev coefficients of 1/Phi in u = 2 (tau/tau_max)^2 - 1
    int deg = 0;
    double inv_tmax2 = 0.0;    // 1 / tau_max^2
    int ppc_pix = 128, ppc_vis = 128;  // points per spreading CTA (bin size), <= 128
    // FP64 plans whose FFT grids go through the double-float FFT: after the FFT the grid
    // holds float pairs (float4 per cell), which the double-float gathers and crop read.
    bool df_grids = false;
    // FP64 spreading into fixed-point tiles of 32-bit limbs (k_nufft.cu) instead of FP64
    // shared atomics.
    bool int_tile = false;
};

// Stage boundaries reported by the kernel launchers to the executor's profiler.
struct StageHook {
    virtual void begin(int stage, cudaStream_t s) = 0;
    virtual void end(int stage, int launches, cudaStream_t s) = 0;
    virtual ~StageHook() = default;
};

// An execution lane for waves of NUFFT sub-problems: its own stream, grid buffers, cuFFT
// plans and cuFFT work area, so that waves on different lanes run concurrently.
struct Lane {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    DevBuf g1, g2, work;
    std::map<std::tuple<int64_t, int64_t, int64_t, int64_t, int64_t>, FftPlans> fft;  // (n2, half, K)
    ~Lane();
};

// One captured CUDA graph of the middle of a transform (everything between the two
// permutations), for one direction and one profiling state.
struct GraphRun {
    struct Bracket {
        int stage;
        cudaEvent_t a, b;
    };
    cudaGraphExec_t exec = nullptr;
    int64_t launches[HVOX_NUM_STAGES] = {0};  // kernel launches per replay, by stage
    std::vector<Bracket> brackets;            // stage brackets (profiled variant: event nodes)
    std::vector<cudaEvent_t> owned;           // events referenced by the event nodes
    cudaEvent_t done = nullptr;               // recorded after a profiled replay
    bool outstanding = false;                 // a profiled replay not yet read back
    ~GraphRun();
};

struct Plan {
    // statistics
    bool profiling = false;
    bool serial = false;   // profiling mode 2: every stage on the plan's stream, one at a time
    double stage_ms[HVOX_NUM_STAGES] = {0};
    int64_t stage_launches[HVOX_NUM_STAGES] = {0};
    int64_t transforms = 0;
    struct Pending {
        int stage;
        cudaEvent_t a, b;
    };
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> event_pool;

    // configuration
    int64_t n_pix = 0, n_vis = 0;
    double eps = 0;
    int isign = -1;
    int prec = 1;          // 1 fp32, 2 fp64
    int mode = 0;
    bool plain = false;
    bool direct_f64 = false;       // direct sums by the FP64 kernels (plain form, or eps < 1e-9)
    int ntrans = 1;
    int direct_vpt = 2;            // points per thread of the direct kernels (owner tile 256 * vpt)
    double sigma = 2.0;
    double budget_opt = 0.0;       // chunk_budget_bytes option (0 -> cost-model search)
    bool sigma_auto = true;        // upsampling chosen by the planner
    double eps_es = 1e-6;          // tolerance given to the kernel-width rule
    double direct_threshold = 0.0; // direct_threshold option
    double search_threshold = 0.01; // search_threshold option (seconds)
    int factor = 0;                // factor option
    bool autotune = false;         // autotune option
    int fixed_w = 0;               // kernel_width option (0: the width rule)
    double probe_error = -1.0;     // measured error of the chosen width on the autotuner's probe
    int ppc_pix = 128, ppc_vis = 128;  // points per spreading CTA (bin size) of each direction
    ESKernel es;
    bool has_weight = false;
    cudaStream_t stream = nullptr;
    int device = 0;

    PartitionResult part;
    double plan_seconds = 0;

    // chunk-ordered geometry
    DevBuf pix_perm, vis_perm;          // int32 position -> original index
    DevBuf weight;                      // double[n_pix] chunk order (or empty)
    DevBuf pix_xyz, vis_xyz;            // double SoA [3][n] chunk order
    DevBuf pix_hi, pix_lo, vis_hi, vis_lo;  // float4 splits of the FP64 coordinates

    // direct work lists
    DevBuf items_s2v, items_v2s;
    DevBuf item_counter;                // int[2]: work-item counters of the direct launches
    int64_t n_items_s2v = 0, n_items_v2s = 0;
    std::vector<WorkItem> host_items[2];  // the same lists on the host (merged batch launches)
    cudaEvent_t batch_event = nullptr;  // orders a batch call against the plan's own stream

    // NUFFT sub-problems
    DevBuf inv_psi;                     // T per (block, dim, l): 1 / Psi on the n1 band
    DevBuf cheb;                        // T: Chebyshev coefficients of 1/Phi
    int cheb_deg = 0;
    double cheb_inv_tmax2 = 0.0;
    std::vector<std::unique_ptr<Lane>> lanes;  // NUFFT execution lanes
    cudaEvent_t fork_event = nullptr;   // main stream -> lanes
    std::vector<NufftDev> dblocks;      // block descriptors (wave order)
    DevBuf ddescs;                      // the same descriptors on the device
    std::vector<Wave> waves;            // waves of blocks (launch order)
    std::map<int, std::unique_ptr<DevBuf>> dfft_tw;  // twiddle tables of the double-float FFT
    bool df_grids = false;              // every FFT batch double-float (NufftArgs::df_grids)
    bool int_tile = false;              // NufftArgs::int_tile
    DevBuf cis_tab;                     // exp(j 2 pi m / 2048) as float pairs (double-float path)
    DevBuf err;                         // int: device error word (kDevErr* bits), read by hvox_sync

    // per-call buffers (chunk order)
    DevBuf src, acc;                    // source values, accumulated outputs
    DevBuf io_in, io_out;               // staging for host-pointer calls
    DevBuf cplx_sky, cplx_vis;          // complex-sky calls: two real skies, one visibility set

    // CUDA graphs (per direction, per profiling state)
    bool chunk_order = false;           // hvox_opts.chunk_order: caller data already in chunk order
    int graphs_opt = 0;                 // hvox_opts.graphs
    int graph_state = 0;                // 0 eager so far, 1 captured, -1 capture failed
    int eager_calls[2] = {0, 0};
    cudaStream_t cap = nullptr;         // capture stream
    std::unique_ptr<GraphRun> graph[2][2];

    double workspace_bytes = 0;
    ~Plan();
};

// ------------------------------------------------------------------ kernel launchers

// Split FP64 (n, 3) coordinates into hi/lo float4 arrays and an FP64 SoA copy, in chunk
// order given perm (position -> original index).
void launch_prepare_points(const double *xyz_orig_dev, const int32_t *perm, int64_t n, double *soa,
                           float4 *hi, float4 *lo, cudaStream_t s);
void launch_gather_weight(const double *w_orig_dev, const int32_t *perm, int64_t n, double *w_perm,
                          cudaStream_t s);

// Direct kernels (k_direct.cu). Owner tile = direct_tile() points per work item.
int direct_tile(int vpt);
void launch_direct_s2v_f32(const WorkItem *items, int64_t n, int *counter, const float4 *vh, const float4 *vl, const float4 *rh,
                           const float4 *rl, const float *c, float2 *acc, int isign, int vpt, cudaStream_t s);
void launch_direct_s2v_df(const WorkItem *items, int64_t n, int *counter, const float4 *vh, const float4 *vl, const float4 *rh,
                          const float4 *rl, const double *c, double2 *acc, const float4 *tab, int isign,
                          int vpt, cudaStream_t s);
void launch_direct_s2v_f64(const WorkItem *items, int64_t n, int *counter, const double *vxyz, int64_t nv, const double *pxyz,
                           int64_t np, const double *c, double2 *acc, int isign, int vpt, cudaStream_t s);
void launch_direct_v2s_f32(const WorkItem *items, int64_t n, int *counter, const float4 *rh, const float4 *rl, const float4 *vh,
                           const float4 *vl, const float2 *V, float *acc, int isign, int vpt, cudaStream_t s);
void launch_direct_v2s_df(const WorkItem *items, int64_t n, int *counter, const float4 *rh, const float4 *rl, const float4 *vh,
                          const float4 *vl, const double2 *V, double *acc, const float4 *tab, int isign,
                          int vpt, cudaStream_t s);
void launch_direct_v2s_f64(const WorkItem *items, int64_t n, int *counter, const double *pxyz, int64_t np, const double *vxyz,
                           int64_t nv, const double2 *V, double *acc, int isign, int vpt, cudaStream_t s);
// Several jobs' items in one launch: kind 0 FP32, 1 double-float; dir 0 sky -> vis, 1 vis -> sky.
void launch_direct_batch(int kind, int dir, const WorkItem *items, int64_t n, int *counter, const DirectJob *jobs,
                         const int *item_job, const float4 *tab, int vpt, cudaStream_t s);

// NUFFT sub-problems, one wave at a time (k_nufft.cu). g1 / g2: the lane's grid buffers.
template <typename T>
void nufft_wave_s2v(const Wave &w, const NufftArgs<T> &a, void *g1, void *g2, const T *c,
                    typename CplxOf<T>::type *acc, cudaStream_t s, StageHook &hook);
template <typename T>
void nufft_wave_v2s(const Wave &w, const NufftArgs<T> &a, void *g1, void *g2, const typename CplxOf<T>::type *V,
                    T *acc, cudaStream_t s, StageHook &hook);

// Device time (ms) of the spreading launch of wave w with ppc points per CTA: pixels onto
// the n1 grids (pix) or baselines onto the n2 grids, values c / V (the grids are cleared
// first, untimed).
template <typename T>
float time_spread(const Wave &w, const NufftArgs<T> &a, void *g1, void *g2, bool pix, const void *values, int ppc,
                  cudaStream_t s);

// Permutations between the caller's order and chunk order (k_misc.cu).
void launch_s2v_in(int prec, const void *I, const int32_t *perm, const double *w, int64_t n, void *src, cudaStream_t s);
void launch_s2v_out(int prec, const void *acc, const int32_t *perm, int64_t n, void *V, cudaStream_t s);
void launch_v2s_in(int prec, const void *V, const int32_t *perm, int64_t n, void *src, cudaStream_t s);
void launch_v2s_out(int prec, const void *acc, const int32_t *perm, const double *w, int64_t n, void *I, cudaStream_t s);

// Plan-wide kernel arguments of the NUFFT launchers (grids and FFT plans set per block).
template <typename T> NufftArgs<T> plan_nufft_args(const Plan &p);

// Transforms.
void run_synthesize(Plan &p, const void *I_dev, void *V_dev);
void run_analyze(Plan &p, const void *V_dev, void *I_dev);
// Complex sky (device pointers, ntrans = 1): two real transforms combined by linearity.
void run_synthesize_complex(Plan &p, const void *I_dev, void *V_dev);
void run_analyze_complex(Plan &p, const void *V_dev, void *I_dev);
void launch_split_complex(int prec, const void *z, int64_t n, void *re, void *im, cudaStream_t s);
void launch_join_complex(int prec, const void *re, const void *im, int64_t n, void *z, cudaStream_t s);
void launch_add_j(int prec, void *a, const void *b, int64_t n, cudaStream_t s);
void launch_times_mj(int prec, const void *a, int64_t n, void *out, cudaStream_t s);
void collect_stats(Plan &p);
// Transforms of several distinct plans (ntrans = 1, device pointers) on stream s, direction
// dir (0 sky -> vis, 1 vis -> sky), with the direct sums of the plans that use the FP32 or
// the double-float kernels merged into one launch per kernel form. Returns the number of
// direct-sum launches made.
int run_batch(const std::vector<Plan *> &plans, const std::vector<const void *> &in, const std::vector<void *> &out,
              int dir, cudaStream_t s);
// Reads (and clears) the device error word after the plan's stream has been synchronised;
// a set word fails with HVOX_EINTERNAL.
void check_device_error(Plan &p);

}  // namespace hvox
