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
                                      p.n_pix, p.src.as<double>(), p.acc.as<double2>(), p.isign, s);
            else if (p.prec == 1)
                launch_direct_s2v_f32(it, p.n_items_s2v, p.vis_hi.as<float4>(), p.vis_lo.as<float4>(),
                                      p.pix_hi.as<float4>(), p.pix_lo.as<float4>(), p.src.as<float>(),
                                      p.acc.as<float2>(), p.isign, s);
            else
                launch_direct_s2v_df(it, p.n_items_s2v, p.vis_hi.as<float4>(), p.vis_lo.as<float4>(),
                                     p.pix_hi.as<float4>(), p.pix_lo.as<float4>(), p.src.as<double>(),
                                     p.acc.as<double2>(), p.cis_tab.as<float4>(), p.isign, s);
            prof.end(HVOX_STAGE_DIRECT, 1);
        }
        for (size_t b = 0; b < p.dblocks.size(); ++b) {
            const DevBlock &db = p.dblocks[b];
            cufftHandle fh = p.block_fft[b];
            if (p.prec == 1)
                nufft_block_s2v<float>(db, p.es.w, p.es.beta, p.src.as<float>(), p.pix_rec.as<GridRec<float>>(),
                                       p.pix_phase.as<float2>(), p.vis_rec.as<GridRec<float>>(),
                                       p.vis_phase.as<float2>(), p.inv_psi.as<float>() + db.psi_off,
                                       p.grid1.as<float2>(), p.grid2.as<float2>(), fh, p.isign, p.acc.as<float2>(), s,
                                       prof);
            else
                nufft_block_s2v<double>(db, p.es.w, p.es.beta, p.src.as<double>(), p.pix_rec.as<GridRec<double>>(),
                                        p.pix_phase.as<double2>(), p.vis_rec.as<GridRec<double>>(),
                                        p.vis_phase.as<double2>(), p.inv_psi.as<double>() + db.psi_off,
                                        p.grid1.as<double2>(), p.grid2.as<double2>(), fh, p.isign,
                                        p.acc.as<double2>(), s, prof);
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
                                      p.n_vis, p.src.as<double2>(), p.acc.as<double>(), p.isign, s);
            else if (p.prec == 1)
                launch_direct_v2s_f32(it, p.n_items_v2s, p.pix_hi.as<float4>(), p.pix_lo.as<float4>(),
                                      p.vis_hi.as<float4>(), p.vis_lo.as<float4>(), p.src.as<float2>(),
                                      p.acc.as<float>(), p.isign, s);
            else
                launch_direct_v2s_df(it, p.n_items_v2s, p.pix_hi.as<float4>(), p.pix_lo.as<float4>(),
                                     p.vis_hi.as<float4>(), p.vis_lo.as<float4>(), p.src.as<double2>(),
                                     p.acc.as<double>(), p.cis_tab.as<float4>(), p.isign, s);
            prof.end(HVOX_STAGE_DIRECT, 1);
        }
        for (size_t b = 0; b < p.dblocks.size(); ++b) {
            const DevBlock &db = p.dblocks[b];
            cufftHandle fh = p.block_fft[b];
            if (p.prec == 1)
                nufft_block_v2s<float>(db, p.es.w, p.es.beta, p.src.as<float2>(), p.pix_rec.as<GridRec<float>>(),
                                       p.pix_phase.as<float2>(), p.vis_rec.as<GridRec<float>>(),
                                       p.vis_phase.as<float2>(), p.inv_psi.as<float>() + db.psi_off,
                                       p.grid1.as<float2>(), p.grid2.as<float2>(), fh, p.isign, p.acc.as<float>(), s,
                                       prof);
            else
                nufft_block_v2s<double>(db, p.es.w, p.es.beta, p.src.as<double2>(),
                                        p.pix_rec.as<GridRec<double>>(), p.pix_phase.as<double2>(),
                                        p.vis_rec.as<GridRec<double>>(), p.vis_phase.as<double2>(),
                                        p.inv_psi.as<double>() + db.psi_off, p.grid1.as<double2>(),
                                        p.grid2.as<double2>(), fh, p.isign, p.acc.as<double>(), s, prof);
        }
        prof.begin(HVOX_STAGE_PERMUTE);
        launch_v2s_out(p.prec, p.acc.ptr, p.pix_perm.as<int32_t>(), weight_ptr(p), p.n_pix, It, s);
        prof.end(HVOX_STAGE_PERMUTE, 1);
        p.transforms++;
    }
}

}  // namespace hvox
