// C ABI of libhvox: argument checking, plan construction (host planner + device
// tables), transform entry points and introspection. Every entry point converts
// internal failures into a status code and a thread-local message.
#include <cuda_runtime.h>
#include <cufft.h>

#include <algorithm>
#include <chrono>
#include <numeric>
#include <tuple>
#include <cstdlib>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "hvox_internal.h"

namespace hvox {

namespace {
thread_local std::string g_last_error;
}

void set_error(const std::string &msg) { g_last_error = msg; }
const char *get_error() { return g_last_error.c_str(); }

void fail(hvox_status code, const std::string &msg) { throw Error{code, msg}; }

void check_cuda(cudaError_t e, const char *what) {
    if (e != cudaSuccess) {
        if (e == cudaErrorMemoryAllocation) fail(HVOX_ENOMEM, std::string(what) + ": out of device memory");
        fail(HVOX_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
    }
}

void check_cufft(cufftResult r, const char *what) {
    if (r != CUFFT_SUCCESS) {
        if (r == CUFFT_ALLOC_FAILED) fail(HVOX_ENOMEM, std::string(what) + ": cuFFT allocation failed");
        fail(HVOX_ECUDA, std::string(what) + ": cuFFT error " + std::to_string((int)r));
    }
}

bool fault_hit(const char *site) {
    static std::mutex mu;
    static std::string spec;
    static std::map<std::string, int64_t> seen;
    const char *v = std::getenv("HVOX_FAULT");
    std::lock_guard<std::mutex> lock(mu);
    const std::string now = v ? v : "";
    if (now != spec) {
        spec = now;
        seen.clear();
    }
    if (spec.empty()) return false;
    size_t pos = 0;
    while (pos <= spec.size()) {
        size_t end = spec.find(',', pos);
        if (end == std::string::npos) end = spec.size();
        const std::string item = spec.substr(pos, end - pos);
        const size_t colon = item.find(':');
        if (colon != std::string::npos && item.compare(0, colon, site) == 0) {
            const int64_t n = std::atoll(item.c_str() + colon + 1);
            return ++seen[site] == n;
        }
        pos = end + 1;
    }
    return false;
}

void DevBuf::alloc(size_t n) {
    free_();
    if (n == 0) return;
    if (fault_hit("alloc")) fail(HVOX_ENOMEM, "cudaMalloc of " + std::to_string(n) + " bytes failed (injected)");
    cudaError_t e = cudaMalloc(&ptr, n);
    if (e != cudaSuccess) {
        ptr = nullptr;
        cudaGetLastError();
        fail(HVOX_ENOMEM, "cudaMalloc of " + std::to_string(n) + " bytes failed");
    }
    bytes = n;
}

void DevBuf::free_() {
    if (ptr) cudaFree(ptr);
    ptr = nullptr;
    bytes = 0;
}

Lane::~Lane() {
    if (stream) cudaStreamSynchronize(stream);
    for (auto &kv : fft)
        for (cufftHandle h : {kv.second.full, kv.second.xy, kv.second.z})
            if (h) cufftDestroy(h);
    if (done) cudaEventDestroy(done);
    if (stream) cudaStreamDestroy(stream);
}

GraphRun::~GraphRun() {
    if (exec) cudaGraphExecDestroy(exec);
    for (cudaEvent_t e : owned) cudaEventDestroy(e);
    if (done) cudaEventDestroy(done);
}

Plan::~Plan() {
    cudaStreamSynchronize(stream);
    for (auto &d : graph)
        for (auto &g : d) g.reset();
    if (cap) cudaStreamDestroy(cap);
    lanes.clear();
    if (fork_event) cudaEventDestroy(fork_event);
    if (batch_event) cudaEventDestroy(batch_event);
    for (auto &q : pending) {
        cudaEventDestroy(q.a);
        cudaEventDestroy(q.b);
    }
    for (cudaEvent_t e : event_pool) cudaEventDestroy(e);
}

void check_device_error(Plan &p) {
    if (!p.err.ptr) return;
    int word = 0;
    check_cuda(cudaMemcpy(&word, p.err.ptr, sizeof(int), cudaMemcpyDeviceToHost), "read device error word");
    if (word == 0) return;
    check_cuda(cudaMemset(p.err.ptr, 0, sizeof(int)), "clear device error word");
    std::string what;
    if (word & kDevErrPixWindow) what += " a pixel window fell outside its sub-problem's n1 grid;";
    if (word & kDevErrVisWindow) what += " a baseline window fell beyond one period of its n2 grid;";
    fail(HVOX_EINTERNAL, "device error word " + std::to_string(word) + ":" + what +
                             " the kernels clamped it into the grid, so the transforms since the last check are wrong");
}

namespace {

template <typename F> hvox_status guard(F &&f) {
    try {
        f();
        g_last_error.clear();
        return HVOX_OK;
    } catch (const Error &e) {
        g_last_error = e.msg;
        return e.code;
    } catch (const std::bad_alloc &) {
        g_last_error = "host allocation failed";
        return HVOX_ENOMEM;
    } catch (const std::exception &e) {
        g_last_error = std::string("internal error: ") + e.what();
        return HVOX_EINTERNAL;
    }
}

bool is_device_ptr(const void *p) {
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

void to_host(const double *src, size_t n, std::vector<double> &dst) {
    dst.resize(n);
    if (is_device_ptr(src))
        check_cuda(cudaMemcpy(dst.data(), src, n * sizeof(double), cudaMemcpyDeviceToHost), "copy input to host");
    else
        std::memcpy(dst.data(), src, n * sizeof(double));
}

// Concurrent execution lanes for waves of NUFFT sub-problems, and the grid bytes of one
// wave (a lane holds the grids of its largest wave and a cuFFT work area of about the same
// size, so a plan's NUFFT memory stays below 2 x 2 x 16 GiB).
constexpr int kMaxLanes = 2;
constexpr double kWaveBytes = 16.0 * 1024 * 1024 * 1024;

// Tolerance given to the kernel-width rule: the type-3 transform chains two
// approximations (spread on n1, interpolate on n2), each held to eps. FP32 plans use eps
// itself (their errors sit near the FP32 grids' rounding floor). FP64 plans take a tenth
// of it, one or two cells more kernel width: the ES error bound holds per output against
// the sum of |source| (it grows with the number of sources when measured as relative l2),
// and at eps 1e-9 the bare rule measured 5.8e-9 sky -> vis on 810,000 pixels.
constexpr double kEpsMarginF32 = 1.0;
constexpr double kEpsMarginF64 = 0.1;

// The double-float direct sums carry ~3e-10 of rounding (the exp(j 2 pi f) table's lo
// parts and the phase are FP32-rounded at ~1e-10 turn); below this tolerance the direct
// sums use the FP64 kernels.
constexpr double kDoubleFloatMinEps = 1e-9;

// FP64 plans transform their grids with the double-float FFT (k_dffft.cu) unless eps is
// below 1e-11 (beyond its ~48-bit significands) or the plan is the plain FP64 form; each
// grid shape must also be one it covers. The cost model prices plans by this rule alone.
constexpr double kDfftMinEps = 1e-11;
bool dfft_wanted(int prec, bool plain, double eps) { return prec == 2 && !plain && eps >= kDfftMinEps; }

// HVOX_DF_FFT=0 runs the same plan's FP64 grids through cuFFT Z2Z instead (comparisons).
bool dfft_switched_off() {
    const char *v = std::getenv("HVOX_DF_FFT");
    return v && std::atoi(v) == 0;
}

void upload(DevBuf &b, const void *host, size_t bytes, cudaStream_t s) {
    b.alloc(bytes);
    if (bytes) check_cuda(cudaMemcpyAsync(b.ptr, host, bytes, cudaMemcpyHostToDevice, s), "upload");
}

void build_items(const std::vector<DirectRect> &rects, bool owner_is_vis, int vpt, std::vector<WorkItem> &items) {
    const int64_t T = direct_tile(vpt);
    double work = 0;
    for (auto &r : rects) work += (double)(r.p1 - r.p0) * (double)(r.v1 - r.v0);
    // About 32 items per resident CTA (152 SMs x 4), taken dynamically by the kernels
    // largest first: a launch then ends within a fraction of an item of its ideal time.
    const double target_items = 152.0 * 4.0 * 32.0;
    int64_t seg = (int64_t)std::ceil(work / ((double)T * target_items) / 256.0) * 256;
    seg = std::max<int64_t>(seg, 2048);
    for (auto &r : rects) {
        int64_t o0 = owner_is_vis ? r.v0 : r.p0, o1 = owner_is_vis ? r.v1 : r.p1;
        int64_t s0 = owner_is_vis ? r.p0 : r.v0, s1 = owner_is_vis ? r.p1 : r.v1;
        for (int64_t o = o0; o < o1; o += T)
            for (int64_t q = s0; q < s1; q += seg)
                items.push_back(WorkItem{(int32_t)o, (int32_t)std::min(o + T, o1), (int32_t)q,
                                         (int32_t)std::min(q + seg, s1)});
    }
    std::stable_sort(items.begin(), items.end(), [](const WorkItem &x, const WorkItem &y) {
        return (int64_t)(x.o1 - x.o0) * (x.s1 - x.s0) > (int64_t)(y.o1 - y.o0) * (y.s1 - y.s0);
    });
}

// Autotuned bin size: the points a spreading CTA takes (32, 64 or 128) trade the size of
// its shared tile (the bounding box of their windows) against the tile's set-up and flush
// per point. Each direction's spreading of the wave holding the sub-problem with the most
// points of that set is timed with every candidate (after one untimed launch each) and the
// fastest kept; the values are ones, so the flush writes every touched cell.
template <typename T> void tune_bins(Plan &p) {
    NufftArgs<T> a = plan_nufft_args<T>(p);
    size_t wp = 0, wv = 0;
    for (size_t w = 0; w < p.waves.size(); ++w) {
        if (p.waves[w].max_np > p.waves[wp].max_np) wp = w;
        if (p.waves[w].max_nv > p.waves[wv].max_nv) wv = w;
    }
    const size_t n = p.src.bytes / sizeof(T);
    std::vector<T> ones(n, T(1));
    check_cuda(cudaMemcpy(p.src.ptr, ones.data(), n * sizeof(T), cudaMemcpyHostToDevice), "autotune values");
    for (int pix = 1; pix >= 0; --pix) {
        const Wave &w = p.waves[pix ? wp : wv];
        if ((pix ? w.max_np : w.max_nv) == 0) continue;
        Lane &l = *p.lanes[w.lane];
        int best = 128;
        float best_ms = INFINITY;
        for (int ppc : {128, 64, 32}) {
            time_spread<T>(w, a, l.g1.ptr, l.g2.ptr, pix != 0, p.src.ptr, ppc, p.stream);
            const float ms = time_spread<T>(w, a, l.g1.ptr, l.g2.ptr, pix != 0, p.src.ptr, ppc, p.stream);
            if (ms < best_ms * 0.97f) {  // a smaller bin must win clearly
                best_ms = ms;
                best = ppc;
            }
        }
        (pix ? p.ppc_pix : p.ppc_vis) = best;
    }
}

// The sums of a probe sub-problem (host coordinates) through the library itself, with
// seeded values in [0, 1): V (complex, host) of sky -> vis.
std::vector<double> probe_sums(const hvox_opts &o, const std::vector<double> &pix, const std::vector<double> &uvw,
                               int prec, int isign) {
    const int64_t np = (int64_t)pix.size() / 3, nv = (int64_t)uvw.size() / 3;
    hvox_plan_t h = nullptr;
    if (hvox_plan(pix.data(), np, uvw.data(), nv, nullptr, prec == 1 ? 1e-6 : 1e-9, isign, &o, &h) != HVOX_OK)
        fail(HVOX_EINTERNAL, std::string("autotune probe plan: ") + get_error());
    std::vector<double> out(2 * nv);
    uint64_t state = 0x9E3779B97F4A7C15ull;
    auto next = [&] {  // splitmix64 -> [0, 1)
        uint64_t z = (state += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return (double)((z ^ (z >> 31)) >> 11) * 0x1.0p-53;
    };
    hvox_status st;
    if (prec == 1) {
        std::vector<float> I(np), V(2 * nv);
        for (auto &x : I) x = (float)next();
        st = hvox_synthesize(h, I.data(), V.data());
        for (int64_t k = 0; k < 2 * nv; ++k) out[k] = V[k];
    } else {
        std::vector<double> I(np);
        for (auto &x : I) x = next();
        st = hvox_synthesize(h, I.data(), out.data());
    }
    const std::string msg = get_error();
    hvox_destroy(h);
    if (st != HVOX_OK) fail(HVOX_EINTERNAL, "autotune probe transform: " + msg);
    return out;
}

// Autotuned kernel width: the width rule of Barnett, Magland and af Klinteberg is an upper
// bound. The NUFFT sub-problem with the most points is taken as a probe (its pixels, and
// up to 2,048 of its baselines evenly spaced), evaluated by direct sums of the plan's
// precision (FP32 ~1e-7, double-float ~3e-10) and by a single type-3 NUFFT at the planned
// upsampling with widths w_rule - 2 and w_rule - 1; the narrowest whose relative l2 error
// is within 2.5 eps (a quarter of the bound the plan answers for, which sums many
// sub-problems) is kept, else the rule's width. The measured error is kept for the plan
// info.
int tune_width(Plan &p, const std::vector<double> &pix, const std::vector<double> &uvw) {
    const PartitionResult &part = p.part;
    size_t bi = 0;
    for (size_t i = 1; i < part.blocks.size(); ++i) {
        const NufftBlock &a = part.blocks[i], &b = part.blocks[bi];
        if ((a.p1 - a.p0) + (a.v1 - a.v0) > (b.p1 - b.p0) + (b.v1 - b.v0)) bi = i;
    }
    const NufftBlock &b = part.blocks[bi];
    std::vector<double> ppix, puvw;
    for (int64_t m = b.p0; m < b.p1; ++m)
        for (int d = 0; d < 3; ++d) ppix.push_back(pix[3 * part.pix_perm[m] + d]);
    const int64_t nv = b.v1 - b.v0, take = std::min<int64_t>(nv, 2048);
    for (int64_t t = 0; t < take; ++t) {
        const int64_t m = b.v0 + t * nv / take;
        for (int d = 0; d < 3; ++d) puvw.push_back(uvw[3 * part.vis_perm[m] + d]);
    }
    hvox_opts o;
    std::memset(&o, 0, sizeof(o));
    o.precision = p.prec;
    o.graphs = -1;
    o.stream = p.stream;
    o.mode = HVOX_MODE_DIRECT;
    const std::vector<double> ref = probe_sums(o, ppix, puvw, p.prec, p.isign);
    double nref = 0.0;
    for (double x : ref) nref += x * x;
    auto rel_err = [&](const std::vector<double> &v) {
        double e = 0.0;
        for (size_t k = 0; k < v.size(); ++k) e += (v[k] - ref[k]) * (v[k] - ref[k]);
        return nref > 0.0 ? std::sqrt(e / nref) : std::sqrt(e);
    };
    o.mode = HVOX_MODE_NUFFT;
    o.upsampfac = part.sigma;
    o.chunk_budget_bytes = 1e15;  // one sub-problem
    const double tol = 2.5 * std::max(p.eps, 1e-12);
    const int rule = part.es.w;
    for (int w = std::max(2, rule - 2); w <= rule; ++w) {
        o.kernel_width = w;
        const double err = rel_err(probe_sums(o, ppix, puvw, p.prec, p.isign));
        if (err <= tol || w == rule) {
            p.probe_error = err;
            return w;
        }
    }
    return rule;
}

void build_plan(Plan &p, const double *pix_in, const double *uvw_in, const double *w_in) {
    auto t0 = std::chrono::steady_clock::now();
    cudaStream_t s = p.stream;
    std::vector<double> pix, uvw, wt;
    to_host(pix_in, (size_t)p.n_pix * 3, pix);
    to_host(uvw_in, (size_t)p.n_vis * 3, uvw);
    for (double v : pix)
        if (!std::isfinite(v)) fail(HVOX_EINVAL, "hvox_plan: non-finite pixel coordinate");
    for (double v : uvw)
        if (!std::isfinite(v)) fail(HVOX_EINVAL, "hvox_plan: non-finite baseline coordinate");
    if (w_in) {
        to_host(w_in, (size_t)p.n_pix, wt);
        for (double v : wt)
            if (!std::isfinite(v)) fail(HVOX_EINVAL, "hvox_plan: non-finite weight");
    }

    const int elem = p.prec == 1 ? 8 : 16;
    PlanInputs in{pix.data(), uvw.data(), p.n_pix, p.n_vis, p.sigma, p.es};
    in.prec = p.prec;
    in.mode = p.mode;
    in.plain = p.plain;
    in.direct_f64 = p.direct_f64;
    in.z2z_fft = !dfft_wanted(p.prec, p.plain, p.eps);
    in.budget = p.budget_opt;
    in.direct_threshold = p.direct_threshold;
    in.search_threshold = p.search_threshold;
    in.elem_bytes = elem;
    in.sigma_auto = p.sigma_auto;
    in.eps_es = p.eps_es;
    in.factor = p.factor;
    in.fixed_w = p.fixed_w;
    {
        // Up to kMaxLanes lanes each hold the grids of a wave (at least one sub-problem's)
        // and a cuFFT work area of about the same size: keep that within a third of the
        // free memory.
        size_t free_b = 0, total_b = 0;
        check_cuda(cudaMemGetInfo(&free_b, &total_b), "cudaMemGetInfo");
        in.max_budget = (double)free_b / (3.0 * 2.0 * kMaxLanes);
    }
    p.part = make_partition(in);
    if (p.autotune && !p.fixed_w && !p.plain && !p.part.blocks.empty()) {
        // Measured kernel width: re-plan at the chosen upsampling with a narrower kernel
        // when the probe sub-problem meets the tolerance with it.
        const int w = tune_width(p, pix, uvw);
        if (w != p.part.es.w) {
            in.fixed_w = w;
            in.sigma = p.part.sigma;
            in.es = es_with_width(w, in.sigma);
            in.sigma_auto = false;
            p.part = make_partition(in);
        }
    }
    PartitionResult &part = p.part;
    p.sigma = part.sigma;
    p.es = part.es;

    // Chunk-ordered geometry.
    std::vector<int32_t> pp(p.n_pix), vp(p.n_vis);
    for (int64_t i = 0; i < p.n_pix; ++i) pp[i] = (int32_t)part.pix_perm[i];
    for (int64_t i = 0; i < p.n_vis; ++i) vp[i] = (int32_t)part.vis_perm[i];
    upload(p.pix_perm, pp.data(), pp.size() * 4, s);
    upload(p.vis_perm, vp.data(), vp.size() * 4, s);
    {
        DevBuf tmp;
        upload(tmp, pix.data(), pix.size() * 8, s);
        p.pix_xyz.alloc((size_t)p.n_pix * 3 * 8);
        p.pix_hi.alloc((size_t)p.n_pix * 16);
        p.pix_lo.alloc((size_t)p.n_pix * 16);
        launch_prepare_points(tmp.as<double>(), p.pix_perm.as<int32_t>(), p.n_pix, p.pix_xyz.as<double>(),
                              p.pix_hi.as<float4>(), p.pix_lo.as<float4>(), s);
        check_cuda(cudaStreamSynchronize(s), "prepare pixels");
    }
    {
        DevBuf tmp;
        upload(tmp, uvw.data(), uvw.size() * 8, s);
        p.vis_xyz.alloc((size_t)p.n_vis * 3 * 8);
        p.vis_hi.alloc((size_t)p.n_vis * 16);
        p.vis_lo.alloc((size_t)p.n_vis * 16);
        launch_prepare_points(tmp.as<double>(), p.vis_perm.as<int32_t>(), p.n_vis, p.vis_xyz.as<double>(),
                              p.vis_hi.as<float4>(), p.vis_lo.as<float4>(), s);
        check_cuda(cudaStreamSynchronize(s), "prepare baselines");
    }
    if (w_in) {
        DevBuf tmp;
        upload(tmp, wt.data(), wt.size() * 8, s);
        p.weight.alloc((size_t)p.n_pix * 8);
        launch_gather_weight(tmp.as<double>(), p.pix_perm.as<int32_t>(), p.n_pix, p.weight.as<double>(), s);
        check_cuda(cudaStreamSynchronize(s), "gather weights");
        p.has_weight = true;
    }

    // Direct work lists.
    {
        std::vector<WorkItem> a, b;
        build_items(part.rects, true, p.direct_vpt, a);
        build_items(part.rects, false, p.direct_vpt, b);
        p.item_counter.alloc(2 * sizeof(int));
        p.err.alloc(sizeof(int));
        check_cuda(cudaMemsetAsync(p.err.ptr, 0, sizeof(int), s), "clear device error word");
        upload(p.items_s2v, a.data(), a.size() * sizeof(WorkItem), s);
        upload(p.items_v2s, b.data(), b.size() * sizeof(WorkItem), s);
        p.n_items_s2v = (int64_t)a.size();
        p.n_items_v2s = (int64_t)b.size();
        p.host_items[0] = std::move(a);
        p.host_items[1] = std::move(b);
    }

    // exp(j 2 pi m / 2048), m = 0 .. 2047, split into float pairs (double-float direct path).
    {
        std::vector<float> tab(2048 * 4);
        for (int i = 0; i < 2048; ++i) {
            double ang = 2.0 * M_PI * (double)i / 2048.0;
            double c = std::cos(ang), sn = std::sin(ang);
            float ch = (float)c, sh = (float)sn;
            tab[4 * i + 0] = ch;
            tab[4 * i + 1] = (float)(c - (double)ch);
            tab[4 * i + 2] = sh;
            tab[4 * i + 3] = (float)(sn - (double)sh);
        }
        upload(p.cis_tab, tab.data(), tab.size() * 4, s);
    }

    // NUFFT sub-problems.
    const size_t re = p.prec == 1 ? 4 : 8;
    int64_t psi_total = 0, max_m1 = 0, max_m2 = 0;
    for (auto &b : part.blocks) {
        b.psi_off = psi_total;
        psi_total += b.n1[0] + b.n1[1] + b.n1[2];
        max_m1 = std::max<int64_t>(max_m1, b.n1[0] * b.n1[1] * b.n1[2]);
        max_m2 = std::max<int64_t>(max_m2, b.n2[0] * b.n2[1] * b.n2[2]);
    }
    if (!part.blocks.empty()) {
        // 1 / Psi on the n1 band of each block and dimension.
        std::vector<double> ipsi(psi_total);
        for (auto &b : part.blocks)
            for (int d = 0, off = 0; d < 3; off += (int)b.n1[d], ++d) {
                std::vector<double> xi(b.n1[d]), ft(b.n1[d]);
                for (int64_t l = 0; l < b.n1[d]; ++l) xi[l] = 2.0 * M_PI * (double)(l - b.n1[d] / 2) / (double)b.n2[d];
                es_ft(p.es, xi.data(), b.n1[d], ft.data());
                for (int64_t l = 0; l < b.n1[d]; ++l) ipsi[b.psi_off + off + l] = 1.0 / ft[l];
            }
        // 1 / Phi(tau) for |tau| <= pi / sigma as a Chebyshev series in u = 2 (tau/tau_max)^2 - 1.
        const double tmax = M_PI / p.sigma * 1.001;
        std::vector<double> cheb;
        fit_inv_phi(p.es, tmax, p.prec == 1 ? 1e-9 : 1e-13, cheb);
        p.cheb_deg = (int)cheb.size() - 1;
        p.cheb_inv_tmax2 = 1.0 / (tmax * tmax);
        if (p.prec == 1) {
            std::vector<float> f(ipsi.begin(), ipsi.end()), c(cheb.begin(), cheb.end());
            upload(p.inv_psi, f.data(), f.size() * 4, s);
            upload(p.cheb, c.data(), c.size() * 4, s);
        } else {
            upload(p.inv_psi, ipsi.data(), ipsi.size() * 8, s);
            upload(p.cheb, cheb.data(), cheb.size() * 8, s);
        }
        // Waves: sub-problems of one grid shape (identical n1 and n2: their FFTs batch)
        // are kept together, shapes in order of total cost, and packed into waves whose
        // grids fit the wave budget; the plain form runs one sub-problem per wave.
        // Waves go longest-first to the least-loaded of (up to) two lanes.
        const double elem_b = 2.0 * (double)re;
        auto m1_of = [](const NufftBlock &b) { return b.n1[0] * b.n1[1] * b.n1[2]; };
        auto m2_of = [](const NufftBlock &b) { return b.n2[0] * b.n2[1] * b.n2[2]; };
        auto shape_key = [](const NufftBlock &b) {
            return std::make_tuple(b.n2[0], b.n2[1], b.n2[2], b.n1[0], b.n1[1], b.n1[2]);
        };
        std::map<decltype(shape_key(part.blocks[0])), std::vector<size_t>> buckets;
        for (size_t i = 0; i < part.blocks.size(); ++i) buckets[shape_key(part.blocks[i])].push_back(i);
        std::vector<std::pair<double, std::vector<size_t>>> shapes;
        for (auto &kv : buckets) {
            double c = 0;
            for (size_t i : kv.second) c += part.blocks[i].cost;
            shapes.push_back({c, kv.second});
        }
        std::stable_sort(shapes.begin(), shapes.end(), [](const auto &x, const auto &y) { return x.first > y.first; });
        size_t free_b = 0, total_b = 0;
        check_cuda(cudaMemGetInfo(&free_b, &total_b), "cudaMemGetInfo");
        // A caller-fixed chunk budget also caps a wave's grids (the plan's memory then stays
        // within the budget per lane, as with one sub-problem per lane).
        double wave_cap = p.plain ? 0.0 : std::min((double)free_b / 12.0, kWaveBytes);
        if (p.budget_opt > 0 && !p.plain) wave_cap = std::min(wave_cap, p.budget_opt);
        if (const char *v = std::getenv("HVOX_WAVE_BYTES")) wave_cap = std::atof(v);
        std::vector<size_t> order;              // blocks in wave order
        std::vector<std::pair<int, int>> wb;    // (first, count) of each wave in `order`
        double wave_bytes = 0;
        for (auto &sh : shapes)
            for (size_t i : sh.second) {
                const double bytes = elem_b * (double)(m1_of(part.blocks[i]) + m2_of(part.blocks[i]));
                if (wb.empty() || wave_bytes + bytes > wave_cap) {
                    wb.push_back({(int)order.size(), 0});
                    wave_bytes = 0;
                }
                order.push_back(i);
                wb.back().second++;
                wave_bytes += bytes;
            }
        int n_lanes = (int)std::min<size_t>(2, wb.size());
        if (const char *v = std::getenv("HVOX_NUFFT_LANES")) n_lanes = std::max(1, std::min(n_lanes, std::atoi(v)));
        std::vector<double> load(n_lanes, 0.0);
        std::vector<int64_t> lane_m1(n_lanes, 0), lane_m2(n_lanes, 0);
        for (auto &f : wb) {
            Wave w;
            w.b0 = f.first;
            w.nb = f.second;
            for (int k = 0; k < w.nb; ++k) {
                const NufftBlock &bk = part.blocks[order[w.b0 + k]];
                w.g1_cells += m1_of(bk);
                w.g2_cells += m2_of(bk);
                w.max_np = std::max<int64_t>(w.max_np, bk.p1 - bk.p0);
                w.max_nv = std::max<int64_t>(w.max_nv, bk.v1 - bk.v0);
                w.max_rows1 = std::max<int64_t>(w.max_rows1, bk.n1[1] * bk.n1[2]);
                w.max_rows2 = std::max<int64_t>(w.max_rows2, bk.n2[1] * bk.n2[2]);
                w.cost += bk.cost;
            }
            p.waves.push_back(w);
        }
        {
            std::vector<size_t> by_cost(p.waves.size());
            std::iota(by_cost.begin(), by_cost.end(), 0);
            std::stable_sort(by_cost.begin(), by_cost.end(),
                             [&](size_t x, size_t y) { return p.waves[x].cost > p.waves[y].cost; });
            for (size_t wi : by_cost) {
                Wave &w = p.waves[wi];
                w.lane = (int)(std::min_element(load.begin(), load.end()) - load.begin());
                load[w.lane] += w.cost;
                lane_m1[w.lane] = std::max<int64_t>(lane_m1[w.lane], w.g1_cells);
                lane_m2[w.lane] = std::max<int64_t>(lane_m2[w.lane], w.g2_cells);
            }
        }
        check_cuda(cudaEventCreateWithFlags(&p.fork_event, cudaEventDisableTiming), "cudaEventCreate");
        const cufftType type = p.prec == 1 ? CUFFT_C2C : CUFFT_Z2Z;
        for (int l = 0; l < n_lanes; ++l) {
            auto lane = std::make_unique<Lane>();
            check_cuda(cudaStreamCreateWithFlags(&lane->stream, cudaStreamNonBlocking), "cudaStreamCreate");
            check_cuda(cudaEventCreateWithFlags(&lane->done, cudaEventDisableTiming), "cudaEventCreate");
            lane->g1.alloc((size_t)lane_m1[l] * 2 * re);
            lane->g2.alloc((size_t)lane_m2[l] * 2 * re);
            p.lanes.push_back(std::move(lane));
        }
        // Descriptors in wave order: each sub-problem's n1 grid back to back in its lane's g1,
        // its FFT grid in the interleaved layout of its shape's batch in the lane's g2.
        // cuFFT plans per lane, shape and batch size, one work area per lane. HVOX_FFT_PRUNE=0
        // selects full 3-D plans instead of the pruned pair.
        bool prune = true;
        if (const char *v = std::getenv("HVOX_FFT_PRUNE")) prune = std::atoi(v) != 0;
        const bool use_dfft = dfft_wanted(p.prec, p.plain, p.eps) && !dfft_switched_off();
        std::vector<size_t> max_ws(n_lanes, 0);
        auto make = [&](cufftHandle &h, int rank, long long *n, long long *emb, long long stride, long long dist,
                        long long batch, size_t &ws) {
            check_cufft(cufftCreate(&h), "cufftCreate");  // h lives in the lane's map: the lane destroys it
            if (fault_hit("cufft")) fail(HVOX_ECUDA, "cufftMakePlanMany64: cuFFT error (injected)");
            check_cufft(cufftSetAutoAllocation(h, 0), "cufftSetAutoAllocation");
            check_cufft(cufftMakePlanMany64(h, rank, n, emb, stride, dist, emb, stride, dist, type, batch, &ws),
                        "cufftMakePlanMany64");
        };
        auto split = [](double x, float &h, float &l) {
            h = (float)x;
            l = (float)(x - (double)h);
        };
        // Double-float FFT only when it covers every grid shape of the plan, so that the
        // grids of every wave share one format after the FFT.
        p.df_grids = use_dfft && prune;
        for (const NufftBlock &bk : part.blocks) p.df_grids = p.df_grids && dfft_supported(bk.n2);
        p.dblocks.resize(order.size());
        for (Wave &w : p.waves) {
            Lane &lane = *p.lanes[w.lane];
            char *g2 = static_cast<char *>(lane.g2.ptr);
            int64_t off1 = 0, off2 = 0;  // cells into the lane's g1 / g2
            for (int k = 0; k < w.nb;) {
                // one batch: the run of sub-problems of this shape
                const NufftBlock &first = part.blocks[order[w.b0 + k]];
                int K = 1;
                while (k + K < w.nb && shape_key(part.blocks[order[w.b0 + k + K]]) == shape_key(first)) ++K;
                FftBatch fb;
                fb.g2 = g2 + (size_t)off2 * 2 * re;
                for (int d = 0; d < 3; ++d) fb.n2[d] = first.n2[d];
                fb.half = first.n1[2] / 2;
                fb.K = K;
                fb.h1y = first.n1[1] / 2;
                const int64_t plane = first.n2[0] * first.n2[1];
                // FP64 grids: the double-float FFT on the FP32 pipes where it covers the shape.
                fb.df = p.df_grids;
                if (fb.df) {
                    DfftDev *dd[3] = {&fb.dx, &fb.dy, &fb.dz};
                    for (int q = 0; q < 3; ++q) {
                        const int n = (int)fb.n2[q];
                        dfft_factor(n, *dd[q]);
                        auto &tab = p.dfft_tw[n];
                        if (!tab) {
                            std::vector<float> t;
                            dfft_twiddles(n, t);
                            tab = std::make_unique<DevBuf>();
                            upload(*tab, t.data(), t.size() * sizeof(float), s);
                        }
                        dd[q]->tw = tab->as<float4>();
                    }
                }
                auto key = std::make_tuple(fb.n2[0], fb.n2[1], fb.n2[2], prune ? fb.half : (int64_t)-1, (int64_t)K);
                if (!fb.df && !lane.fft.count(key)) {
                    FftPlans &f = lane.fft[key];
                    size_t ws = 0;
                    if (prune) {
                        long long nxy[2] = {fb.n2[1], fb.n2[0]};
                        make(f.xy, 2, nxy, nullptr, 1, plane, fb.half * K, ws);
                        max_ws[w.lane] = std::max(max_ws[w.lane], ws);
                        long long nz[1] = {fb.n2[2]}, emb[1] = {fb.n2[2]};
                        make(f.z, 1, nz, emb, plane * K, 1, plane * K, ws);
                    } else {
                        long long n3[3] = {fb.n2[2], fb.n2[1], fb.n2[0]};
                        long long e3[3] = {fb.n2[2], fb.n2[1] * K, fb.n2[0]};
                        make(f.full, 3, n3, e3, 1, plane, K, ws);
                    }
                    max_ws[w.lane] = std::max(max_ws[w.lane], ws);
                }
                if (!fb.df) fb.plans = lane.fft[key];
                w.ffts.push_back(fb);
                for (int g = 0; g < K; ++g, ++k) {
                    const NufftBlock &bk = part.blocks[order[w.b0 + k]];
                    NufftDev d;
                    std::memset(&d, 0, sizeof(d));
                    d.p0 = bk.p0;
                    d.np = bk.p1 - bk.p0;
                    d.v0 = bk.v0;
                    d.nv = bk.v1 - bk.v0;
                    for (int q = 0; q < 3; ++q) {
                        d.n1[q] = (int32_t)bk.n1[q];
                        d.n2[q] = (int32_t)bk.n2[q];
                        d.C[q] = bk.C[q];
                        d.D[q] = bk.D[q];
                        d.a[q] = bk.a[q];
                        d.n2a[q] = bk.a[q] > 0 ? (double)bk.n2[q] / bk.a[q] : 0.0;
                        d.tpa64[q] = bk.a[q] > 0 ? 2.0 * M_PI / bk.a[q] : 0.0;
                        split(bk.C[q], d.Ch[q], d.Cl[q]);
                        split(bk.D[q], d.Dh[q], d.Dl[q]);
                        split(bk.a[q], d.ah[q], d.al[q]);
                        split(d.n2a[q], d.n2ah[q], d.n2al[q]);
                        d.tpa[q] = (float)d.tpa64[q];
                    }
                    d.psi_off = bk.psi_off;
                    d.err = p.err.as<int>();
                    d.g1_off = off1;
                    off1 += m1_of(bk);
                    d.g2_off = off2 + (int64_t)g * plane;
                    d.zs2 = plane * K;
                    p.dblocks[w.b0 + k] = d;
                }
                off2 += (int64_t)K * first.n2[0] * first.n2[1] * first.n2[2];
            }
        }
        for (int l = 0; l < n_lanes; ++l) {
            Lane &lane = *p.lanes[l];
            lane.work.alloc(std::max<size_t>(max_ws[l], 256));
            for (auto &kv : lane.fft)
                for (cufftHandle h : {kv.second.full, kv.second.xy, kv.second.z})
                    if (h) check_cufft(cufftSetWorkArea(h, lane.work.ptr), "cufftSetWorkArea");
        }
        if (fault_hit("window")) {  // the sub-problem with the most pixels (a pixel extent to scale)
            NufftDev &d = *std::max_element(p.dblocks.begin(), p.dblocks.end(),
                                            [](const NufftDev &x, const NufftDev &y) { return x.np < y.np; });
            for (int q = 0; q < 3; ++q) {
                d.a[q] *= 4.0;
                split(d.a[q], d.ah[q], d.al[q]);
            }
        }
        upload(p.ddescs, p.dblocks.data(), p.dblocks.size() * sizeof(NufftDev), s);
    }

    // Per-call buffers.
    size_t src_bytes = std::max((size_t)p.n_pix * re, (size_t)p.n_vis * 2 * re);
    p.src.alloc(src_bytes);
    p.acc.alloc(src_bytes);
    check_cuda(cudaStreamSynchronize(s), "hvox_plan");
    if (p.autotune && !p.dblocks.empty()) {
        if (p.prec == 1)
            tune_bins<float>(p);
        else
            tune_bins<double>(p);
    }

    double ws = 0;
    for (DevBuf *b : {&p.pix_perm, &p.vis_perm, &p.weight, &p.pix_xyz, &p.vis_xyz, &p.pix_hi, &p.pix_lo, &p.vis_hi,
                      &p.vis_lo, &p.items_s2v, &p.items_v2s, &p.item_counter, &p.inv_psi, &p.cheb, &p.src, &p.acc, &p.cis_tab, &p.err})
        ws += (double)b->bytes;
    for (auto &l : p.lanes) ws += (double)(l->g1.bytes + l->g2.bytes + l->work.bytes);
    for (auto &kv : p.dfft_tw) ws += (double)kv.second->bytes;
    p.workspace_bytes = ws;
    p.plan_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

// Checks the options and fills the configuration fields of a plan.
void configure(Plan &p, int64_t n_pix, int64_t n_vis, double eps, int isign, const hvox_opts *opts) {
    hvox_opts o;
    std::memset(&o, 0, sizeof(o));
    if (opts) o = *opts;
    if (o.precision < 0 || o.precision > 2) fail(HVOX_EINVAL, "hvox_plan: bad precision");
    if (o.mode < 0 || o.mode > 2) fail(HVOX_EINVAL, "hvox_plan: bad mode");
    if (!(o.upsampfac == 0.0 || (o.upsampfac >= 1.25 && o.upsampfac <= 4.0)))
        fail(HVOX_EINVAL, "hvox_plan: upsampfac must be 0 or in [1.25, 4]");
    if (!(o.chunk_budget_bytes >= 0.0) || !std::isfinite(o.chunk_budget_bytes))
        fail(HVOX_EINVAL, "hvox_plan: bad chunk_budget_bytes");
    if (!(o.anisotropy == 0.0 || o.anisotropy >= 1.0)) fail(HVOX_EINVAL, "hvox_plan: anisotropy must be >= 1");
    if (o.ntrans < 0) fail(HVOX_EINVAL, "hvox_plan: ntrans must be >= 0");
    if (!std::isfinite(o.direct_threshold)) fail(HVOX_EINVAL, "hvox_plan: bad direct_threshold");
    if (!(o.search_threshold >= 0.0) || !std::isfinite(o.search_threshold))
        fail(HVOX_EINVAL, "hvox_plan: bad search_threshold");
    if (o.factor < 0 || o.factor > 2) fail(HVOX_EINVAL, "hvox_plan: factor must be 0, 1 or 2");
    p.factor = o.factor;
    if (o.autotune < 0 || o.autotune > 1) fail(HVOX_EINVAL, "hvox_plan: autotune must be 0 or 1");
    p.autotune = o.autotune != 0;
    if (o.kernel_width != 0 && (o.kernel_width < 2 || o.kernel_width > 16))
        fail(HVOX_EINVAL, "hvox_plan: kernel_width must be 0 or in [2, 16]");
    p.fixed_w = o.kernel_width;
    p.n_pix = n_pix;
    p.n_vis = n_vis;
    p.eps = eps;
    p.isign = isign;
    p.plain = o.plain != 0;
    if (o.graphs < -1 || o.graphs > 1) fail(HVOX_EINVAL, "hvox_plan: graphs must be -1, 0 or 1");
    p.graphs_opt = o.graphs;
    if (o.chunk_order < 0 || o.chunk_order > 1) fail(HVOX_EINVAL, "hvox_plan: chunk_order must be 0 or 1");
    p.chunk_order = o.chunk_order != 0;
    p.mode = eps == 0.0 ? HVOX_MODE_DIRECT : o.mode;
    p.prec = p.plain ? 2 : (o.precision == HVOX_PREC_AUTO ? (eps >= 1e-6 ? 1 : 2) : o.precision);
    p.ntrans = o.ntrans > 0 ? o.ntrans : 1;
    p.sigma = o.upsampfac > 0 ? o.upsampfac : 2.0;
    p.sigma_auto = !(o.upsampfac > 0);
    p.stream = (cudaStream_t)o.stream;
    p.budget_opt = o.chunk_budget_bytes;
    p.direct_threshold = o.direct_threshold;
    p.search_threshold = o.search_threshold > 0 ? o.search_threshold : 0.01;
    double e = eps > 0 ? eps : 1e-6;
    if (p.prec == 1 && e < 1e-7) fail(HVOX_EUNSUPPORTED, "hvox_plan: FP32 cannot reach eps < 1e-7");
    p.eps_es = e * (p.prec == 1 ? kEpsMarginF32 : kEpsMarginF64);
    p.direct_f64 = p.plain || (p.prec == 2 && e < kDoubleFloatMinEps);
    p.es = p.fixed_w ? es_with_width(p.fixed_w, p.sigma) : es_params_within(p.eps_es, e, p.sigma);
    // Fixed-point spreading tiles for FP64 plans (not the plain form); HVOX_SPREAD_TILE=float
    // keeps FP64 shared atomics (comparisons).
    p.int_tile = p.prec == 2 && !p.plain;
    if (const char *v = std::getenv("HVOX_SPREAD_TILE")) p.int_tile = p.int_tile && std::string(v) != "float";
    // Owners per thread of the direct kernels: four for the double-float kernels (LOFAR-like
    // sky x 1.4M baselines at eps 1e-9: 320.2 against 327.8 ms per step), two for the FP32
    // ones (config 2 at eps 1e-6: 125.3 against 126.8 ms) and the FP64 ones. HVOX_DIRECT_VPT
    // (2 or 4) overrides.
    p.direct_vpt = (p.prec == 2 && !p.direct_f64) ? 4 : 2;
    if (const char *v = std::getenv("HVOX_DIRECT_VPT")) p.direct_vpt = std::atoi(v) == 4 ? 4 : 2;
}

void fill_info(const Plan &p, hvox_info *info) {
    std::memset(info, 0, sizeof(*info));
    info->n_pix = p.n_pix;
    info->n_vis = p.n_vis;
    info->precision = p.prec;
    info->isign = p.isign;
    info->eps = p.eps;
    info->w = p.es.w;
    info->beta = p.es.beta;
    info->upsampfac = p.sigma;
    info->budget_bytes = p.part.budget;
    info->t = p.part.t;
    for (int d = 0; d < 3; ++d) {
        info->h[d] = p.part.h[d];
        info->eta[d] = p.part.eta[d];
    }
    info->n_pix_chunks = p.part.n_pix_chunks;
    info->n_vis_chunks = p.part.n_vis_chunks;
    info->n_nufft_blocks = (int64_t)p.part.blocks.size();
    info->n_direct_rects = (int64_t)p.part.rects.size();
    info->direct_pairs = p.part.direct_pairs;
    info->nufft_points = p.part.nufft_points;
    info->nufft_cells = p.part.nufft_cells;
    info->max_grid_bytes = p.part.max_grid_bytes;
    info->workspace_bytes = p.workspace_bytes;
    info->plan_seconds = p.plan_seconds;
    info->model_seconds = p.part.model_seconds;
    info->graph_state = p.graph_state;
    info->nufft_pix_points = p.part.nufft_pix_points;
    info->nufft_vis_points = p.part.nufft_vis_points;
    info->spread_cells = p.part.spread_cells;
    info->fft_work = p.part.fft_work;
    info->box_ratio = p.part.box_ratio;
    info->spread_bin_pix = p.ppc_pix;
    info->spread_bin_vis = p.ppc_vis;
    info->kernel_width_rule = es_params_within(p.eps_es, p.eps > 0 ? p.eps : 1e-6, p.sigma).w;
    info->probe_error = p.probe_error;
    info->direct_vpt = p.direct_vpt;
    info->fft_batches = info->fft_batches_df = 0;
    for (const Wave &w : p.waves)
        for (const FftBatch &f : w.ffts) {
            ++info->fft_batches;
            info->fft_batches_df += f.df ? 1 : 0;
        }
}

void transform(Plan &p, const void *in, void *out, bool s2v) {
    check_cuda(cudaSetDevice(p.device), "cudaSetDevice");
    const size_t re = p.prec == 1 ? 4 : 8;
    const size_t in_bytes = (size_t)p.ntrans * (s2v ? (size_t)p.n_pix * re : (size_t)p.n_vis * 2 * re);
    const size_t out_bytes = (size_t)p.ntrans * (s2v ? (size_t)p.n_vis * 2 * re : (size_t)p.n_pix * re);
    const bool din = is_device_ptr(in), dout = is_device_ptr(out);
    const void *src = in;
    void *dst = out;
    if (!din) {
        size_t need = (size_t)p.ntrans * std::max((size_t)p.n_pix * re, (size_t)p.n_vis * 2 * re);
        if (p.io_in.bytes < need) p.io_in.alloc(need);
        check_cuda(cudaMemcpyAsync(p.io_in.ptr, in, in_bytes, cudaMemcpyHostToDevice, p.stream), "copy input");
        src = p.io_in.ptr;
    }
    if (!dout) {
        size_t need = (size_t)p.ntrans * std::max((size_t)p.n_pix * re, (size_t)p.n_vis * 2 * re);
        if (p.io_out.bytes < need) p.io_out.alloc(need);
        dst = p.io_out.ptr;
    }
    if (s2v)
        run_synthesize(p, src, dst);
    else
        run_analyze(p, src, dst);
    if (!dout) {
        check_cuda(cudaMemcpyAsync(out, dst, out_bytes, cudaMemcpyDeviceToHost, p.stream), "copy output");
        check_cuda(cudaStreamSynchronize(p.stream), "transform");
        check_device_error(p);
    } else if (!din) {
        check_cuda(cudaStreamSynchronize(p.stream), "transform");
        check_device_error(p);
    }
}

}  // namespace
}  // namespace hvox

using namespace hvox;

struct hvox_plan_s {
    Plan p;
};

extern "C" {

const char *hvox_last_error(void) { return get_error(); }

const char *hvox_version(void) { return "hvox-gb300 0.1.0 (sm_103a)"; }

hvox_status hvox_plan(const double *pix_xyz, int64_t n_pix, const double *uvw, int64_t n_vis,
                      const double *pix_weight, double eps, int isign, const hvox_opts *opts, hvox_plan_t *out) {
    if (out) *out = nullptr;
    return guard([&] {
        if (!out) fail(HVOX_EINVAL, "hvox_plan: out is NULL");
        if (!pix_xyz || !uvw) fail(HVOX_EINVAL, "hvox_plan: NULL coordinates");
        if (n_pix < 1 || n_vis < 1) fail(HVOX_EINVAL, "hvox_plan: need n_pix >= 1 and n_vis >= 1");
        if (n_pix > INT32_MAX - 1024 || n_vis > INT32_MAX - 1024) fail(HVOX_EINVAL, "hvox_plan: too many points");
        if (!std::isfinite(eps) || eps < 0.0) fail(HVOX_EINVAL, "hvox_plan: eps must be finite and >= 0");
        if (isign != 1 && isign != -1) fail(HVOX_EINVAL, "hvox_plan: isign must be +1 or -1");
        auto *h = new hvox_plan_s();
        try {
            Plan &p = h->p;
            check_cuda(cudaGetDevice(&p.device), "cudaGetDevice");
            configure(p, n_pix, n_vis, eps, isign, opts);
            build_plan(p, pix_xyz, uvw, pix_weight);
        } catch (...) {
            delete h;
            throw;
        }
        *out = h;
    });
}

hvox_status hvox_synthesize(hvox_plan_t plan, const void *I, void *V) {
    return guard([&] {
        if (!plan || !I || !V) fail(HVOX_EINVAL, "hvox_synthesize: NULL argument");
        transform(plan->p, I, V, true);
    });
}

hvox_status hvox_analyze(hvox_plan_t plan, const void *V, void *I) {
    return guard([&] {
        if (!plan || !I || !V) fail(HVOX_EINVAL, "hvox_analyze: NULL argument");
        transform(plan->p, V, I, false);
    });
}

namespace {
hvox_status batch_call(const hvox_plan_t *plans, const void *const *in, void *const *out, int32_t n, void *stream,
                       int32_t *direct_launches, int dir) {
    const char *name = dir == 0 ? "hvox_synthesize_batch" : "hvox_analyze_batch";
    return guard([&] {
        if (direct_launches) *direct_launches = 0;
        if (n < 0 || (n > 0 && (!plans || !in || !out))) fail(HVOX_EINVAL, std::string(name) + ": NULL argument");
        if (n == 0) return;
        std::vector<Plan *> ps((size_t)n);
        std::vector<const void *> ins((size_t)n);
        std::vector<void *> outs((size_t)n);
        for (int32_t i = 0; i < n; ++i) {
            if (!plans[i] || !in[i] || !out[i]) fail(HVOX_EINVAL, std::string(name) + ": NULL plan or buffer");
            ps[i] = &plans[i]->p;
            for (int32_t j = 0; j < i; ++j)
                if (ps[j] == ps[i]) fail(HVOX_EINVAL, std::string(name) + ": a plan appears twice");
            if (ps[i]->device != ps[0]->device) fail(HVOX_EINVAL, std::string(name) + ": plans on different devices");
            if (ps[i]->ntrans != 1) fail(HVOX_EUNSUPPORTED, std::string(name) + ": ntrans must be 1");
            ins[i] = in[i];
            outs[i] = out[i];
        }
        check_cuda(cudaSetDevice(ps[0]->device), "cudaSetDevice");
        for (int32_t i = 0; i < n; ++i)
            if (!is_device_ptr(ins[i]) || !is_device_ptr(outs[i]))
                fail(HVOX_EINVAL, std::string(name) + ": device pointers only");
        const int l = run_batch(ps, ins, outs, dir, static_cast<cudaStream_t>(stream));
        if (direct_launches) *direct_launches = l;
    });
}
}  // namespace

hvox_status hvox_synthesize_batch(const hvox_plan_t *plans, const void *const *I, void *const *V, int32_t n,
                                  void *stream, int32_t *direct_launches) {
    return batch_call(plans, I, V, n, stream, direct_launches, 0);
}

hvox_status hvox_analyze_batch(const hvox_plan_t *plans, const void *const *V, void *const *I, int32_t n,
                               void *stream, int32_t *direct_launches) {
    return batch_call(plans, V, I, n, stream, direct_launches, 1);
}

hvox_status hvox_synthesize_complex(hvox_plan_t plan, const void *I, void *V) {
    return guard([&] {
        if (!plan || !I || !V) fail(HVOX_EINVAL, "hvox_synthesize_complex: NULL argument");
        Plan &p = plan->p;
        check_cuda(cudaSetDevice(p.device), "cudaSetDevice");
        if (p.ntrans != 1) fail(HVOX_EUNSUPPORTED, "hvox_synthesize_complex: ntrans must be 1");
        if (!is_device_ptr(I) || !is_device_ptr(V)) fail(HVOX_EINVAL, "hvox_synthesize_complex: device pointers only");
        run_synthesize_complex(p, I, V);
    });
}

hvox_status hvox_analyze_complex(hvox_plan_t plan, const void *V, void *I) {
    return guard([&] {
        if (!plan || !I || !V) fail(HVOX_EINVAL, "hvox_analyze_complex: NULL argument");
        Plan &p = plan->p;
        check_cuda(cudaSetDevice(p.device), "cudaSetDevice");
        if (p.ntrans != 1) fail(HVOX_EUNSUPPORTED, "hvox_analyze_complex: ntrans must be 1");
        if (!is_device_ptr(I) || !is_device_ptr(V)) fail(HVOX_EINVAL, "hvox_analyze_complex: device pointers only");
        run_analyze_complex(p, V, I);
    });
}

hvox_status hvox_dirty2vis(hvox_plan_t plan, const void *I, void *V) { return hvox_synthesize(plan, I, V); }
hvox_status hvox_vis2dirty(hvox_plan_t plan, const void *V, void *I) { return hvox_analyze(plan, V, I); }

hvox_status hvox_destroy(hvox_plan_t plan) {
    return guard([&] { delete plan; });
}

hvox_status hvox_sync(hvox_plan_t plan) {
    return guard([&] {
        if (!plan) fail(HVOX_EINVAL, "hvox_sync: NULL plan");
        check_cuda(cudaSetDevice(plan->p.device), "cudaSetDevice");
        check_cuda(cudaStreamSynchronize(plan->p.stream), "hvox_sync");
        check_cuda(cudaGetLastError(), "hvox_sync");
        check_device_error(plan->p);
    });
}

hvox_status hvox_profile(hvox_plan_t plan, int enable) {
    return guard([&] {
        if (!plan) fail(HVOX_EINVAL, "hvox_profile: NULL plan");
        Plan &p = plan->p;
        check_cuda(cudaSetDevice(p.device), "cudaSetDevice");
        collect_stats(p);
        for (int i = 0; i < HVOX_NUM_STAGES; ++i) {
            p.stage_ms[i] = 0.0;
            p.stage_launches[i] = 0;
        }
        p.transforms = 0;
        if (enable < 0 || enable > 2) fail(HVOX_EINVAL, "hvox_profile: enable must be 0, 1 or 2");
        p.profiling = enable != 0;
        p.serial = enable == 2;
    });
}

hvox_status hvox_get_stats(hvox_plan_t plan, hvox_stats *out) {
    return guard([&] {
        if (!plan || !out) fail(HVOX_EINVAL, "hvox_get_stats: NULL argument");
        Plan &p = plan->p;
        check_cuda(cudaSetDevice(p.device), "cudaSetDevice");
        collect_stats(p);
        check_cuda(cudaStreamSynchronize(p.stream), "hvox_get_stats");
        check_device_error(p);
        for (int i = 0; i < HVOX_NUM_STAGES; ++i) {
            out->ms[i] = p.stage_ms[i];
            out->launches[i] = p.stage_launches[i];
        }
        out->transforms = p.transforms;
    });
}

hvox_status hvox_plan_info(hvox_plan_t plan, hvox_info *info) {
    return guard([&] {
        if (!plan || !info) fail(HVOX_EINVAL, "hvox_plan_info: NULL argument");
        fill_info(plan->p, info);
    });
}

hvox_status hvox_cost_model(int32_t precision, int32_t plain, double rates[8]) {
    return guard([&] {
        if (!rates) fail(HVOX_EINVAL, "hvox_cost_model: NULL rates");
        if (precision != HVOX_PREC_FP32 && precision != HVOX_PREC_FP64)
            fail(HVOX_EINVAL, "hvox_cost_model: precision must be HVOX_PREC_FP32 or HVOX_PREC_FP64");
        const CostModel m = default_cost_model(precision, plain != 0, 0);
        const double v[8] = {m.direct_pair, m.scatter_smem, m.scatter_global, m.gather_tap,
                             m.fft_cell,    m.grid_cell,    m.block_fixed,    m.tile_cells};
        for (int i = 0; i < 8; ++i) rates[i] = v[i];
    });
}

hvox_status hvox_plan_dry(const double *pix_xyz, int64_t n_pix, const double *uvw, int64_t n_vis, double eps,
                          const hvox_opts *opts, hvox_info *info) {
    return guard([&] {
        if (!pix_xyz || !uvw || !info) fail(HVOX_EINVAL, "hvox_plan_dry: NULL argument");
        if (n_pix < 1 || n_vis < 1) fail(HVOX_EINVAL, "hvox_plan_dry: need n_pix >= 1 and n_vis >= 1");
        if (!std::isfinite(eps) || eps < 0.0) fail(HVOX_EINVAL, "hvox_plan_dry: eps must be finite and >= 0");
        for (int64_t i = 0; i < 3 * n_pix; ++i)
            if (!std::isfinite(pix_xyz[i])) fail(HVOX_EINVAL, "hvox_plan_dry: non-finite pixel coordinate");
        for (int64_t i = 0; i < 3 * n_vis; ++i)
            if (!std::isfinite(uvw[i])) fail(HVOX_EINVAL, "hvox_plan_dry: non-finite baseline coordinate");
        auto t0 = std::chrono::steady_clock::now();
        Plan p;
        configure(p, n_pix, n_vis, eps, -1, opts);
        const int elem = p.prec == 1 ? 8 : 16;
        PlanInputs in{pix_xyz, uvw, n_pix, n_vis, p.sigma, p.es};
        in.prec = p.prec;
        in.mode = p.mode;
        in.plain = p.plain;
        in.direct_f64 = p.direct_f64;
        in.z2z_fft = !dfft_wanted(p.prec, p.plain, p.eps);
        in.budget = p.budget_opt;
        in.direct_threshold = p.direct_threshold;
        in.search_threshold = p.search_threshold;
        in.elem_bytes = elem;
        in.sigma_auto = p.sigma_auto;
        in.eps_es = p.eps_es;
        in.factor = p.factor;
        in.fixed_w = p.fixed_w;
    in.fixed_w = p.fixed_w;
        p.part = make_partition(in);
        p.sigma = p.part.sigma;
        p.es = p.part.es;
        // Estimate of what hvox_plan would allocate: coordinates and permutations, the
        // source and accumulator, and per lane the grids of a wave and a cuFFT work area of
        // about the same size.
        const double re = p.prec == 1 ? 4.0 : 8.0;
        const double lanes = (double)std::min<size_t>(kMaxLanes, p.part.blocks.size());
        const double all_grids = 2.0 * re * (p.part.spread_cells + p.part.nufft_cells);
        const double wave = std::max(p.part.max_grid_bytes, std::min(all_grids, kWaveBytes));
        p.workspace_bytes = (double)(n_pix + n_vis) * 60.0 + 2.0 * lanes * wave +
                            4.0 * re * (double)std::max(n_pix, 2 * n_vis);
        p.plan_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        fill_info(p, info);
    });
}

hvox_status hvox_plan_order(hvox_plan_t plan, int64_t *pix_order, int64_t *vis_order) {
    return guard([&] {
        if (!plan) fail(HVOX_EINVAL, "hvox_plan_order: NULL plan");
        const Plan &p = plan->p;
        if (pix_order) std::memcpy(pix_order, p.part.pix_perm.data(), sizeof(int64_t) * p.n_pix);
        if (vis_order) std::memcpy(vis_order, p.part.vis_perm.data(), sizeof(int64_t) * p.n_vis);
    });
}

hvox_status hvox_plan_chunks(hvox_plan_t plan, int64_t *pix_chunk, int64_t *vis_chunk) {
    return guard([&] {
        if (!plan) fail(HVOX_EINVAL, "hvox_plan_chunks: NULL plan");
        const Plan &p = plan->p;
        if (pix_chunk) std::memcpy(pix_chunk, p.part.pix_label.data(), sizeof(int64_t) * p.n_pix);
        if (vis_chunk) std::memcpy(vis_chunk, p.part.vis_label.data(), sizeof(int64_t) * p.n_vis);
    });
}

double hvox_estimate_bytes(int64_t n_pix, int64_t n_vis, double eps, const hvox_opts *opts) {
    if (n_pix < 1 || n_vis < 1 || !(eps >= 0.0)) return 0.0;
    int prec = 1;
    const bool plain = opts && opts->plain;
    if (plain) prec = 2;
    else if (opts && opts->precision) prec = opts->precision;
    else if (eps > 0 && eps < 1e-6) prec = 2;
    const double re = prec == 1 ? 4.0 : 8.0;
    const int nt = (opts && opts->ntrans > 0) ? opts->ntrans : 1;
    double geom = (double)(n_pix + n_vis) * (4.0 + 24.0 + 32.0) + (double)n_pix * 8.0;
    double bufs = 2.0 * std::max((double)n_pix * re, (double)n_vis * 2.0 * re);
    double io = 2.0 * nt * std::max((double)n_pix * re, (double)n_vis * 2.0 * re);
    // Jobs the planner keeps as direct sums without a search own no NUFFT grids; others
    // own at most kMaxLanes lanes of wave grids and cuFFT work areas, each within the
    // larger of the wave bytes and the chunk budget.
    const CostModel m = default_cost_model(prec, plain || (prec == 2 && eps > 0 && eps < kDoubleFloatMinEps), 0,
                                           !dfft_wanted(prec, plain, eps));
    const double search = (opts && opts->search_threshold > 0) ? opts->search_threshold : 0.01;
    const bool auto_plan = !(opts && (opts->mode != HVOX_MODE_AUTO || opts->direct_threshold > 0 ||
                                      opts->chunk_budget_bytes > 0));
    const bool direct_only = eps == 0.0 || (opts && opts->mode == HVOX_MODE_DIRECT) ||
                             (auto_plan && 2.0 * m.direct_pair * (double)n_pix * (double)n_vis < search);
    const double budget = (opts && opts->chunk_budget_bytes > 0) ? opts->chunk_budget_bytes : 8.0 * 1024 * 1024 * 1024;
    const double wave = (opts && opts->chunk_budget_bytes > 0) ? budget : std::max(budget, kWaveBytes);
    const double grids = direct_only ? 0.0 : 2.0 * kMaxLanes * wave;
    return geom + bufs + io + grids;
}

hvox_status hvox_es_params(double eps, double sigma, int32_t *w, double *beta) {
    return guard([&] {
        if (!w || !beta) fail(HVOX_EINVAL, "hvox_es_params: NULL output");
        ESKernel k = es_params(eps, sigma);
        *w = k.w;
        *beta = k.beta;
    });
}

hvox_status hvox_es_ft(int32_t w, double beta, const double *xi, int64_t n, double *out) {
    return guard([&] {
        if (w < 2 || w > 16 || !(beta > 0) || n < 0 || (n > 0 && (!xi || !out)))
            fail(HVOX_EINVAL, "hvox_es_ft: bad arguments");
        ESKernel k;
        k.w = w;
        k.beta = beta;
        es_ft(k, xi, n, out);
    });
}

hvox_status hvox_box_dims(const double P[3], const double B[3], double budget_bytes, double sigma, int32_t w,
                          int32_t elem_bytes, double eta[3], double h[3], double *t) {
    return guard([&] {
        if (!P || !B || !eta || !h || !t) fail(HVOX_EINVAL, "hvox_box_dims: NULL argument");
        if (!(budget_bytes > 0) || !(sigma > 1.0) || w < 2 || elem_bytes <= 0)
            fail(HVOX_EINVAL, "hvox_box_dims: bad arguments");
        for (int d = 0; d < 3; ++d)
            if (!(P[d] >= 0) || !(B[d] >= 0) || !std::isfinite(P[d]) || !std::isfinite(B[d]))
                fail(HVOX_EINVAL, "hvox_box_dims: extents must be finite and >= 0");
        *t = box_dims(P, B, budget_bytes, sigma, w, elem_bytes, eta, h);
    });
}

hvox_status hvox_chunk_points(const double *xyz, int64_t n, const double h[3], int64_t *labels, int64_t *n_chunks) {
    return guard([&] {
        if (!xyz || !h || !labels || !n_chunks || n < 0) fail(HVOX_EINVAL, "hvox_chunk_points: bad arguments");
        for (int64_t i = 0; i < 3 * n; ++i)
            if (!std::isfinite(xyz[i])) fail(HVOX_EINVAL, "hvox_chunk_points: non-finite coordinate");
        std::vector<int64_t> lab;
        *n_chunks = chunk_points(xyz, n, h, lab);
        if (n) std::memcpy(labels, lab.data(), sizeof(int64_t) * n);
    });
}

}  // extern "C"
