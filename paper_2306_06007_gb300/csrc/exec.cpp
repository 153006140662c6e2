// Executor: one transform = permute in -> direct rectangles -> NUFFT sub-problems ->
// permute out, all enqueued on the plan's stream (Fig. 6 flow: inputs to chunk order,
// sub-transforms, row sums, outputs back to the caller's order).
#include <cuda_runtime.h>

#include "hvox_internal.h"

namespace hvox {

namespace {

size_t real_bytes(const Plan &p) { return p.prec == 1 ? sizeof(float) : sizeof(double); }

const double *weight_ptr(const Plan &p) { return p.has_weight ? p.weight.as<double>() : nullptr; }

cudaEvent_t take_event(Plan &p) {
    if (!p.event_pool.empty()) {
        cudaEvent_t e = p.event_pool.back();
        p.event_pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    check_cuda(cudaEventCreate(&e), "cudaEventCreate");
    return e;
}

// Counts launches per stage and, when profiling, brackets each stage with events on
// the plan's stream.
struct Profiler final : StageHook {
    Plan &p;
    cudaEvent_t open = nullptr;
    explicit Profiler(Plan &plan) : p(plan) {}
    void begin(int) override {
        if (!p.profiling) return;
        open = take_event(p);
        check_cuda(cudaEventRecord(open, p.stream), "cudaEventRecord");
    }
    void end(int stage, int launches) override {
        p.stage_launches[stage] += launches;
        if (!p.profiling || !open) return;
        cudaEvent_t b = take_event(p);
        check_cuda(cudaEventRecord(b, p.stream), "cudaEventRecord");
        p.pending.push_back({stage, open, b});
        open = nullptr;
    }
};

template <typename T> NufftArgs<T> nufft_args(const Plan &p) {
    NufftArgs<T> a;
    a.w = p.es.w;
    a.beta = p.es.beta;
    a.isign = p.isign;
    a.G1 = p.grid1.as<typename CplxOf<T>::type>();
    a.G2 = p.grid2.as<typename CplxOf<T>::type>();
    a.ipsi = p.inv_psi.as<T>();
    a.pix_hi = p.pix_hi.as<float4>();
    a.pix_lo = p.pix_lo.as<float4>();
    a.vis_hi = p.vis_hi.as<float4>();
    a.vis_lo = p.vis_lo.as<float4>();
    a.pix_soa = p.pix_xyz.as<double>();
    a.vis_soa = p.vis_xyz.as<double>();
    a.n_pix = p.n_pix;
    a.n_vis = p.n_vis;
    a.cheb = p.cheb.as<T>();
    a.deg = p.cheb_deg;
    a.inv_tmax2 = p.cheb_inv_tmax2;
    return a;
}

}  // namespace

void collect_stats(Plan &p) {
    if (p.pending.empty()) return;
    check_cuda(cudaStreamSynchronize(p.stream), "collect_stats");
    for (auto &q : p.pending) {
        float ms = 0.f;
        check_cuda(cudaEventElapsedTime(&ms, q.a, q.b), "cudaEventElapsedTime");
        p.stage_ms[q.stage] += ms;
        p.event_pool.push_back(q.a);
        p.event_pool.push_back(q.b);
    }
    p.pending.clear();
}

void run_synthesize(Plan &p, const void *I, void *V) {
    cudaStream_t s = p.stream;
    const size_t re = real_bytes(p);
    Profiler prof(p);
    for (int t = 0; t < p.ntrans; ++t) {
        const char *It = (const char *)I + (size_t)t * p.n_pix * re;
        char *Vt = (char *)V + (size_t)t * p.n_vis * 2 * re;
        prof.begin(HVOX_STAGE_PERMUTE);
        launch_s2v_in(p.prec, It, p.pix_perm.as<int32_t>(), weight_ptr(p), p.n_pix, p.src.ptr, s);
        prof.end(HVOX_STAGE_PERMUTE, 1);
        prof.begin(HVOX_STAGE_ZERO);
        check_cuda(cudaMemsetAsync(p.acc.ptr, 0, (size_t)p.n_vis * 2 * re, s), "memset acc");
        prof.end(HVOX_STAGE_ZERO, 1);
        if (p.n_items_s2v > 0) {
            prof.begin(HVOX_STAGE_DIRECT);
            const WorkItem *it = p.items_s2v.as<WorkItem>();
            if (p.plain)
                launch_direct_s2v_f64(it, p.n_items_s2v, p.vis_xyz.as<double>(), p.n_vis, p.pix_xyz.as<double>(),
                                      p.n_pix, p.src.as<double>(), p.acc.as<double2>(), p.isign, p.direct_vpt, s);
            else if (p.prec == 1)
                launch_direct_s2v_f32(it, p.n_items_s2v, p.vis_hi.as<float4>(), p.vis_lo.as<float4>(),
                                      p.pix_hi.as<float4>(), p.pix_lo.as<float4>(), p.src.as<float>(),
                                      p.acc.as<float2>(), p.isign, p.direct_vpt, s);
            else
                launch_direct_s2v_df(it, p.n_items_s2v, p.vis_hi.as<float4>(), p.vis_lo.as<float4>(),
                                     p.pix_hi.as<float4>(), p.pix_lo.as<float4>(), p.src.as<double>(),
                                     p.acc.as<double2>(), p.cis_tab.as<float4>(), p.isign, p.direct_vpt, s);
            prof.end(HVOX_STAGE_DIRECT, 1);
        }
        if (!p.dblocks.empty()) {
            if (p.prec == 1) {
                NufftArgs<float> a = nufft_args<float>(p);
                for (size_t b = 0; b < p.dblocks.size(); ++b) {
                    a.fft = p.block_fft[b];
                    nufft_block_s2v<float>(p.dblocks[b], a, p.src.as<float>(), p.acc.as<float2>(), s, prof);
                }
            } else {
                NufftArgs<double> a = nufft_args<double>(p);
                for (size_t b = 0; b < p.dblocks.size(); ++b) {
                    a.fft = p.block_fft[b];
                    nufft_block_s2v<double>(p.dblocks[b], a, p.src.as<double>(), p.acc.as<double2>(), s, prof);
                }
            }
        }
        prof.begin(HVOX_STAGE_PERMUTE);
        launch_s2v_out(p.prec, p.acc.ptr, p.vis_perm.as<int32_t>(), p.n_vis, Vt, s);
        prof.end(HVOX_STAGE_PERMUTE, 1);
        p.transforms++;
    }
}

void run_analyze(Plan &p, const void *V, void *I) {
    cudaStream_t s = p.stream;
    const size_t re = real_bytes(p);
    Profiler prof(p);
    for (int t = 0; t < p.ntrans; ++t) {
        const char *Vt = (const char *)V + (size_t)t * p.n_vis * 2 * re;
        char *It = (char *)I + (size_t)t * p.n_pix * re;
        prof.begin(HVOX_STAGE_PERMUTE);
        launch_v2s_in(p.prec, Vt, p.vis_perm.as<int32_t>(), p.n_vis, p.src.ptr, s);
        prof.end(HVOX_STAGE_PERMUTE, 1);
        prof.begin(HVOX_STAGE_ZERO);
        check_cuda(cudaMemsetAsync(p.acc.ptr, 0, (size_t)p.n_pix * re, s), "memset acc");
        prof.end(HVOX_STAGE_ZERO, 1);
        if (p.n_items_v2s > 0) {
            prof.begin(HVOX_STAGE_DIRECT);
            const WorkItem *it = p.items_v2s.as<WorkItem>();
            if (p.plain)
                launch_direct_v2s_f64(it, p.n_items_v2s, p.pix_xyz.as<double>(), p.n_pix, p.vis_xyz.as<double>(),
                                      p.n_vis, p.src.as<double2>(), p.acc.as<double>(), p.isign, p.direct_vpt, s);
            else if (p.prec == 1)
                launch_direct_v2s_f32(it, p.n_items_v2s, p.pix_hi.as<float4>(), p.pix_lo.as<float4>(),
                                      p.vis_hi.as<float4>(), p.vis_lo.as<float4>(), p.src.as<float2>(),
                                      p.acc.as<float>(), p.isign, p.direct_vpt, s);
            else
                launch_direct_v2s_df(it, p.n_items_v2s, p.pix_hi.as<float4>(), p.pix_lo.as<float4>(),
                                     p.vis_hi.as<float4>(), p.vis_lo.as<float4>(), p.src.as<double2>(),
                                     p.acc.as<double>(), p.cis_tab.as<float4>(), p.isign, p.direct_vpt, s);
            prof.end(HVOX_STAGE_DIRECT, 1);
        }
        if (!p.dblocks.empty()) {
            if (p.prec == 1) {
                NufftArgs<float> a = nufft_args<float>(p);
                for (size_t b = 0; b < p.dblocks.size(); ++b) {
                    a.fft = p.block_fft[b];
                    nufft_block_v2s<float>(p.dblocks[b], a, p.src.as<float2>(), p.acc.as<float>(), s, prof);
                }
            } else {
                NufftArgs<double> a = nufft_args<double>(p);
                for (size_t b = 0; b < p.dblocks.size(); ++b) {
                    a.fft = p.block_fft[b];
                    nufft_block_v2s<double>(p.dblocks[b], a, p.src.as<double2>(), p.acc.as<double>(), s, prof);
                }
            }
        }
        prof.begin(HVOX_STAGE_PERMUTE);
        launch_v2s_out(p.prec, p.acc.ptr, p.pix_perm.as<int32_t>(), weight_ptr(p), p.n_pix, It, s);
        prof.end(HVOX_STAGE_PERMUTE, 1);
        p.transforms++;
    }
}

}  // namespace hvox
