// Executor: one transform = permute in -> direct rectangles -> NUFFT sub-problems ->
// permute out, all enqueued on the plan's stream (Fig. 6 flow: inputs to chunk order,
// sub-transforms, row sums, outputs back to the caller's order).
#include <cuda_runtime.h>

#include "hvox_internal.h"

namespace hvox {

namespace {

size_t real_bytes(const Plan &p) { return p.prec == 1 ? sizeof(float) : sizeof(double); }

const double *weight_ptr(const Plan &p) { return p.has_weight ? p.weight.as<double>() : nullptr; }

}  // namespace

void run_synthesize(Plan &p, const void *I, void *V) {
    cudaStream_t s = p.stream;
    const size_t re = real_bytes(p);
    for (int t = 0; t < p.ntrans; ++t) {
        const char *It = (const char *)I + (size_t)t * p.n_pix * re;
        char *Vt = (char *)V + (size_t)t * p.n_vis * 2 * re;
        launch_s2v_in(p.prec, It, p.pix_perm.as<int32_t>(), weight_ptr(p), p.n_pix, p.src.ptr, s);
        check_cuda(cudaMemsetAsync(p.acc.ptr, 0, (size_t)p.n_vis * 2 * re, s), "memset acc");
        if (p.n_items_s2v > 0) {
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
        }
        for (size_t b = 0; b < p.dblocks.size(); ++b) {
            const DevBlock &db = p.dblocks[b];
            cufftHandle fh = p.block_fft[b];
            if (p.prec == 1)
                nufft_block_s2v<float>(db, p.es.w, p.es.beta, p.src.as<float>(), p.pix_rec.as<GridRec<float>>(),
                                       p.pix_phase.as<float2>(), p.vis_rec.as<GridRec<float>>(),
                                       p.vis_phase.as<float2>(), p.inv_psi.as<float>() + db.psi_off,
                                       p.grid1.as<float2>(), p.grid2.as<float2>(), fh, p.isign, p.acc.as<float2>(), s);
            else
                nufft_block_s2v<double>(db, p.es.w, p.es.beta, p.src.as<double>(), p.pix_rec.as<GridRec<double>>(),
                                        p.pix_phase.as<double2>(), p.vis_rec.as<GridRec<double>>(),
                                        p.vis_phase.as<double2>(), p.inv_psi.as<double>() + db.psi_off,
                                        p.grid1.as<double2>(), p.grid2.as<double2>(), fh, p.isign,
                                        p.acc.as<double2>(), s);
        }
        launch_s2v_out(p.prec, p.acc.ptr, p.vis_perm.as<int32_t>(), p.n_vis, Vt, s);
    }
}

void run_analyze(Plan &p, const void *V, void *I) {
    cudaStream_t s = p.stream;
    const size_t re = real_bytes(p);
    for (int t = 0; t < p.ntrans; ++t) {
        const char *Vt = (const char *)V + (size_t)t * p.n_vis * 2 * re;
        char *It = (char *)I + (size_t)t * p.n_pix * re;
        launch_v2s_in(p.prec, Vt, p.vis_perm.as<int32_t>(), p.n_vis, p.src.ptr, s);
        check_cuda(cudaMemsetAsync(p.acc.ptr, 0, (size_t)p.n_pix * re, s), "memset acc");
        if (p.n_items_v2s > 0) {
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
        }
        for (size_t b = 0; b < p.dblocks.size(); ++b) {
            const DevBlock &db = p.dblocks[b];
            cufftHandle fh = p.block_fft[b];
            if (p.prec == 1)
                nufft_block_v2s<float>(db, p.es.w, p.es.beta, p.src.as<float2>(), p.pix_rec.as<GridRec<float>>(),
                                       p.pix_phase.as<float2>(), p.vis_rec.as<GridRec<float>>(),
                                       p.vis_phase.as<float2>(), p.inv_psi.as<float>() + db.psi_off,
                                       p.grid1.as<float2>(), p.grid2.as<float2>(), fh, p.isign, p.acc.as<float>(), s);
            else
                nufft_block_v2s<double>(db, p.es.w, p.es.beta, p.src.as<double2>(),
                                        p.pix_rec.as<GridRec<double>>(), p.pix_phase.as<double2>(),
                                        p.vis_rec.as<GridRec<double>>(), p.vis_phase.as<double2>(),
                                        p.inv_psi.as<double>() + db.psi_off, p.grid1.as<double2>(),
                                        p.grid2.as<double2>(), fh, p.isign, p.acc.as<double>(), s);
        }
        launch_v2s_out(p.prec, p.acc.ptr, p.pix_perm.as<int32_t>(), weight_ptr(p), p.n_pix, It, s);
    }
}

}  // namespace hvox
