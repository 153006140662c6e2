// Host planner: Algorithm 1 (maximum Heisenberg dimensions), Algorithm 2 (chunking),
// the per-sub-problem choice between type-3 NUFFT and direct evaluation (Sect. 3.1,
// last benefit of chunking), the chunk-order permutation (Sect. 4) and the work
// decomposition executed by the kernels.
//
// Readings where the paper is silent:
//  * Algorithm 1 is solved at its isotropic optimum h = t B, eta = t P (optimal for
//    any alpha >= 1, unique at alpha = 1), with the memory budget applied to the
//    padded spread and FFT grids a full-size sub-problem allocates (bisection on t).
//  * Algorithm 2 fusion: lattice cells in lexicographic order; each unassigned
//    occupied cell seeds a chunk and absorbs, in lexicographic offset order, the
//    unassigned occupied cells of the 2x2x2 window at its minimum corner while the
//    chunk's point bounding box stays within h in every dimension.
#include <algorithm>
#include <cmath>
#include <future>
#include <numeric>
#include <thread>

#include "hvox_internal.h"

namespace hvox {

int64_t smooth_even(int64_t n) {
    int64_t m = std::max<int64_t>(2, n);
    if (m % 2) ++m;
    for (;; m += 2) {
        int64_t r = m;
        for (int64_t f : {2, 3, 5, 7})
            while (r % f == 0) r /= f;
        if (r == 1) return m;
    }
}

void grid_sizes(double extent_pix, double extent_vis, double sigma, int w, int64_t &n1, int64_t &n2) {
    double need = sigma * extent_pix * extent_vis + (double)w + 2.0;
    n1 = 2 * (int64_t)std::ceil(need / 2.0);
    n2 = smooth_even(std::max<int64_t>((int64_t)std::ceil(sigma * (double)n1), 2 * (int64_t)w));
}

double grid_bytes(const double P[3], const double B[3], double sigma, int w, int elem_bytes) {
    double n1p = 1, n2p = 1;
    for (int d = 0; d < 3; ++d) {
        int64_t n1, n2;
        grid_sizes(P[d], B[d], sigma, w, n1, n2);
        n1p *= (double)n1;
        n2p *= (double)n2;
    }
    return (double)elem_bytes * (n1p + n2p);
}

double box_dims(const double P[3], const double B[3], double budget, double sigma, int w, int elem_bytes,
                double eta[3], double h[3]) {
    double t;
    if (grid_bytes(P, B, sigma, w, elem_bytes) <= budget) {
        t = 1.0;
    } else {
        double lo = 0.0, hi = 1.0;
        for (int it = 0; it < 64; ++it) {
            double mid = 0.5 * (lo + hi);
            double Pm[3], Bm[3];
            for (int d = 0; d < 3; ++d) {
                Pm[d] = mid * P[d];
                Bm[d] = mid * B[d];
            }
            if (grid_bytes(Pm, Bm, sigma, w, elem_bytes) <= budget)
                lo = mid;
            else
                hi = mid;
        }
        t = lo;
    }
    for (int d = 0; d < 3; ++d) {
        eta[d] = t * P[d];
        h[d] = t * B[d];
    }
    return t;
}

namespace {

struct Key {
    int64_t x, y, z;
    bool operator<(const Key &o) const {
        if (x != o.x) return x < o.x;
        if (y != o.y) return y < o.y;
        return z < o.z;
    }
    bool operator==(const Key &o) const { return x == o.x && y == o.y && z == o.z; }
};

}  // namespace

int64_t chunk_points(const double *xyz, int64_t n, const double h[3], std::vector<int64_t> &labels) {
    labels.assign(n, 0);
    if (n == 0) return 0;
    double lo[3] = {xyz[0], xyz[1], xyz[2]};
    for (int64_t i = 1; i < n; ++i)
        for (int d = 0; d < 3; ++d) lo[d] = std::min(lo[d], xyz[3 * i + d]);
    std::vector<std::pair<Key, int64_t>> kp(n);
    for (int64_t i = 0; i < n; ++i) {
        int64_t c[3] = {0, 0, 0};
        for (int d = 0; d < 3; ++d)
            if (h[d] > 0.0 && std::isfinite(h[d])) c[d] = (int64_t)std::floor((xyz[3 * i + d] - lo[d]) / h[d]);
        kp[i] = {Key{c[0], c[1], c[2]}, i};
    }
    std::sort(kp.begin(), kp.end(), [](const auto &a, const auto &b) {
        if (a.first == b.first) return a.second < b.second;
        return a.first < b.first;
    });
    // Occupied cells (step 3) with their point bounding boxes.
    std::vector<Key> cells;
    std::vector<int64_t> cstart;
    std::vector<double> cbox;  // 6 per cell: lo xyz, hi xyz
    for (int64_t i = 0; i < n; ++i) {
        const double *p = xyz + 3 * kp[i].second;
        if (i == 0 || !(kp[i].first == kp[i - 1].first)) {
            cells.push_back(kp[i].first);
            cstart.push_back(i);
            for (int d = 0; d < 3; ++d) cbox.push_back(p[d]);
            for (int d = 0; d < 3; ++d) cbox.push_back(p[d]);
        } else {
            double *b = &cbox[cbox.size() - 6];
            for (int d = 0; d < 3; ++d) {
                b[d] = std::min(b[d], p[d]);
                b[3 + d] = std::max(b[3 + d], p[d]);
            }
        }
    }
    cstart.push_back(n);
    const int64_t nc = (int64_t)cells.size();
    std::vector<int64_t> owner(nc, -1);
    static const int off[7][3] = {{0, 0, 1}, {0, 1, 0}, {0, 1, 1}, {1, 0, 0}, {1, 0, 1}, {1, 1, 0}, {1, 1, 1}};
    int64_t n_chunks = 0;
    for (int64_t c = 0; c < nc; ++c) {
        if (owner[c] >= 0) continue;
        const int64_t cid = n_chunks++;
        owner[c] = cid;
        double blo[3], bhi[3];
        for (int d = 0; d < 3; ++d) {
            blo[d] = cbox[6 * c + d];
            bhi[d] = cbox[6 * c + 3 + d];
        }
        for (int o = 0; o < 7; ++o) {
            Key nb{cells[c].x + off[o][0], cells[c].y + off[o][1], cells[c].z + off[o][2]};
            auto it = std::lower_bound(cells.begin(), cells.end(), nb);
            if (it == cells.end() || !(*it == nb)) continue;
            int64_t j = it - cells.begin();
            if (owner[j] >= 0) continue;
            double jlo[3], jhi[3];
            bool ok = true;
            for (int d = 0; d < 3; ++d) {
                jlo[d] = std::min(blo[d], cbox[6 * j + d]);
                jhi[d] = std::max(bhi[d], cbox[6 * j + 3 + d]);
                if (!(jhi[d] - jlo[d] <= h[d])) ok = false;
            }
            if (ok) {
                for (int d = 0; d < 3; ++d) {
                    blo[d] = jlo[d];
                    bhi[d] = jhi[d];
                }
                owner[j] = cid;
            }
        }
    }
    for (int64_t c = 0; c < nc; ++c)
        for (int64_t i = cstart[c]; i < cstart[c + 1]; ++i) labels[kp[i].second] = owner[c];
    return n_chunks;
}

CostModel default_cost_model(int prec, bool plain, int w, bool z2z_fft) {
    // Seconds per unit of work on one GB300, measured with this library's kernels: direct
    // pairs/s of the FP32, double-float and FP64 kernels; spreading taps/s through
    // shared-memory tiles and straight into the grid (vector atomics); interpolation
    // taps/s; cuFFT C2C (HBM-bound), the double-float FFT of FP64 grids and cuFFT Z2Z
    // (bound by GB300's FP64 units) per cell and log2(cells); grid passes at HBM speed.
    (void)w;
    CostModel m;
    if (prec == 1 && !plain) {
        // Stage rates fitted by calibrate.py (least squares through the origin over the 1, 3
        // and 10 km sweep cases and the dense-core workload, serial profiling mode,
        // CUDA-event stage times; the fit is stored with the tests). The direct rate is the
        // large launch of the SKA-Low-like benchmark line (2.9e12 pairs per launch), since
        // the calibration workloads have almost no direct work.
        m.direct_pair = 1.0 / 1.17e12;
        m.scatter_smem = 1.0 / 6.3e11;
        m.scatter_global = 1.0 / 2.4e11;
        m.gather_tap = 1.0 / 9.7e11;
        m.fft_cell = 4.1e-13;
        m.grid_cell = 8.8e-13;
        m.block_fixed = 30e-6;
        m.tile_cells = 12000.0;  // shared tile of a spreading CTA (float planes, w <= 8)
    } else {
        // FP64 sub-problems, fitted the same way (calibrate.py --eps 1e-9 --mode nufft, 1 to
        // 40 sub-problems per workload). Spreading taps are one rate: the fit does not
        // separate the shared-tile and global paths (fixed-point tiles, double-float taps
        // and weights; the gathers in double-float arithmetic). The FFT rate is the
        // double-float FFT's (4.2x cheaper per cell than cuFFT Z2Z, which is bound by the
        // FP64 units at ~17x the C2C rate and still serves the plain form and eps < 1e-11,
        // measured earlier). The double-float direct rate is the LOFAR-like benchmark's launch.
        // The plain form keeps FP64 arithmetic in every kernel: its earlier fit (FP64 shared
        // and global atomics, FP64 gathers) stays. The spreading and gather rates sit ~4 %
        // below the least-squares fit (1/2.49e11, 1/3.67e11 s), which the baseline-heavy
        // dense core dominates, toward the faster per-tap rates of the pixel-heavy sweep cases.
        m.direct_pair = plain ? 1.0 / 4.0e9 : 1.0 / 4.6e11;
        m.scatter_smem = plain ? 1.0 / 1.15e11 : 1.0 / 2.60e11;
        m.scatter_global = m.scatter_smem;
        m.gather_tap = plain ? 1.0 / 1.22e11 : 1.0 / 3.80e11;
        m.fft_cell = (plain || z2z_fft) ? 7.2e-12 : 1.7e-12;
        m.grid_cell = 1.7e-12;
        m.block_fixed = 50e-6;
        m.tile_cells = 4800.0;   // double planes, w ~ 10
    }
    return m;
}

namespace {

struct ChunkStats {
    std::vector<int64_t> count;
    std::vector<double> lo, hi;  // 3 per chunk
};

ChunkStats stats_of(const double *xyz, int64_t n, const std::vector<int64_t> &labels, int64_t nc) {
    ChunkStats s;
    s.count.assign(nc, 0);
    s.lo.assign(3 * nc, INFINITY);
    s.hi.assign(3 * nc, -INFINITY);
    for (int64_t i = 0; i < n; ++i) {
        int64_t c = labels[i];
        s.count[c]++;
        for (int d = 0; d < 3; ++d) {
            s.lo[3 * c + d] = std::min(s.lo[3 * c + d], xyz[3 * i + d]);
            s.hi[3 * c + d] = std::max(s.hi[3 * c + d], xyz[3 * i + d]);
        }
    }
    return s;
}

constexpr double kMaxCandidatePairs = 16.0 * 1024.0 * 1024.0;

struct Evaluated {
    double t, h[3], eta[3], budget, ratio = 1.0;
    std::vector<int64_t> pl, vl;
    int64_t npc, nvc;
    ChunkStats ps, vs;
    std::vector<std::pair<int64_t, int64_t>> nufft_pairs;  // (pix chunk, vis chunk)
    double cost = 0.0;
};

// Spreading cost per tap for n points on a grid of `cells`: through the shared tile when
// the 128 points of a CTA (uniform-density estimate of the region they occupy, plus the
// kernel width) fit the tile, else straight into the grid.
double scatter_cost(const CostModel &m, double n, double cells, int w) {
    double region = 128.0 * cells / std::max(1.0, n);
    double side = std::cbrt(region) + (double)(w - 1);
    return side * side * side <= m.tile_cells ? m.scatter_smem : m.scatter_global;
}

// Modelled cost of one sub-problem by NUFFT in both directions (sky -> vis spreads pixels
// and gathers baselines; vis -> sky spreads baselines and gathers pixels).
double nufft_cost(const CostModel &m, const ESKernel &es, double sigma, int64_t np, int64_t nv, const double *pext,
                  const double *vext, double *cells_out) {
    double m1 = 1, m2 = 1;
    for (int d = 0; d < 3; ++d) {
        int64_t n1, n2;
        grid_sizes(pext[d], vext[d], sigma, es.w, n1, n2);
        m1 *= (double)n1;
        m2 *= (double)n2;
    }
    if (cells_out) *cells_out = m2;
    const double w3 = (double)es.w * es.w * es.w;
    const double taps_p = (double)np * w3, taps_v = (double)nv * w3;
    double c = taps_p * (scatter_cost(m, (double)np, m1, es.w) + m.gather_tap) +
               taps_v * (scatter_cost(m, (double)nv, m2, es.w) + m.gather_tap);
    c += 2.0 * (m.fft_cell * m2 * std::log2(std::max(2.0, m2)) + m.grid_cell * (2.0 * m1 + 2.0 * m2) + m.block_fixed);
    return c;
}

// ratio: how the Heisenberg volume of Algorithm 1's boxes is split between the two sets
// (eta scaled by ratio, h by 1 / ratio: the same grid per sub-problem, larger pixel chunks
// and smaller baseline chunks for ratio > 1).
Evaluated evaluate(const PlanInputs &in, const CostModel &m, double budget, const double P[3], const double B[3],
                   double ratio = 1.0) {
    Evaluated e;
    e.budget = budget;
    e.ratio = ratio;
    e.t = box_dims(P, B, budget, in.sigma, in.es.w, in.elem_bytes, e.eta, e.h);
    if (e.t <= 0.0 && in.mode != HVOX_MODE_DIRECT) {
        // the budget cannot hold even the smallest grid (2w cells per dimension)
        e.cost = INFINITY;
        return e;
    }
    if (ratio != 1.0)
        for (int d = 0; d < 3; ++d) {
            e.eta[d] *= ratio;
            e.h[d] /= ratio;
        }
    e.npc = chunk_points(in.pix, in.n_pix, e.eta, e.pl);
    e.nvc = chunk_points(in.uvw, in.n_vis, e.h, e.vl);
    e.ps = stats_of(in.pix, in.n_pix, e.pl, e.npc);
    e.vs = stats_of(in.uvw, in.n_vis, e.vl, e.nvc);
    const double w3 = (double)in.es.w * in.es.w * in.es.w;
    double total = 0.0;
    double direct_pairs = (double)in.n_pix * (double)in.n_vis;
    if (in.mode == HVOX_MODE_DIRECT) {
        e.cost = 2.0 * m.direct_pair * direct_pairs;
        return e;
    }
    // Chunks too small to ever win as NUFFT (tap cost alone exceeds the direct cost).
    double min_pts = (in.mode == HVOX_MODE_NUFFT || in.direct_threshold > 0)
                         ? 0.0
                         : (m.scatter_smem + m.gather_tap) * w3 / (2.0 * m.direct_pair);
    std::vector<int64_t> bigp, bigv;
    for (int64_t i = 0; i < e.npc; ++i)
        if ((double)e.ps.count[i] > min_pts) bigp.push_back(i);
    for (int64_t j = 0; j < e.nvc; ++j)
        if ((double)e.vs.count[j] > min_pts) bigv.push_back(j);
    // A budget so small that the candidate sub-problems number in the tens of millions
    // (forced NUFFT mode at the smallest budgets) is not a plan: it is marked infeasible
    // instead of being enumerated.
    if ((double)bigp.size() * (double)bigv.size() > kMaxCandidatePairs) {
        e.cost = INFINITY;
        return e;
    }
    for (int64_t i : bigp) {
        double pext[3];
        for (int d = 0; d < 3; ++d) pext[d] = e.ps.hi[3 * i + d] - e.ps.lo[3 * i + d];
        for (int64_t j : bigv) {
            double vext[3];
            for (int d = 0; d < 3; ++d) vext[d] = e.vs.hi[3 * j + d] - e.vs.lo[3 * j + d];
            int64_t np = e.ps.count[i], nv = e.vs.count[j];
            double pairs = (double)np * (double)nv;
            bool use_nufft;
            double cn = 0.0;
            if (in.mode == HVOX_MODE_NUFFT) {
                use_nufft = true;
                cn = nufft_cost(m, in.es, in.sigma, np, nv, pext, vext, nullptr);
            } else if (in.direct_threshold > 0) {
                use_nufft = pairs > in.direct_threshold;
                if (use_nufft) cn = nufft_cost(m, in.es, in.sigma, np, nv, pext, vext, nullptr);
            } else {
                cn = nufft_cost(m, in.es, in.sigma, np, nv, pext, vext, nullptr);
                use_nufft = cn < 2.0 * m.direct_pair * pairs;
            }
            if (use_nufft) {
                for (int d = 0; d < 3 && use_nufft; ++d) {
                    int64_t n1, n2;
                    grid_sizes(pext[d], vext[d], in.sigma, in.es.w, n1, n2);
                    if (n2 > 65535 || n1 > 65535) use_nufft = false;  // launch-grid limit
                }
            }
            if (use_nufft) {
                e.nufft_pairs.push_back({i, j});
                total += cn;
                direct_pairs -= pairs;
            }
        }
    }
    total += 2.0 * m.direct_pair * direct_pairs;
    e.cost = total;
    return e;
}

// Box split of a factored evaluation at this budget: factor 1 makes the baseline box span
// every baseline (h = B; pixel boxes shrink by t so that the grid keeps Algorithm 1's size)
// and factor 2 makes the pixel box span the sky (eta = P). A hair of slack keeps the
// extreme points in the first lattice cell. 1 when Algorithm 1's boxes already span both.
double factored_ratio(int factor, const double P[3], const double B[3], double budget, double sigma, int w,
                      int elem_bytes) {
    double eta[3], h[3];
    const double t = box_dims(P, B, budget, sigma, w, elem_bytes, eta, h);
    if (!(t > 0.0) || t >= 1.0) return 1.0;
    return factor == 1 ? t / 1.000001 : 1.000001 / t;
}

}  // namespace

PartitionResult make_partition(const PlanInputs &in) {
    PartitionResult r;
    CostModel m = default_cost_model(in.prec, in.plain, in.es.w, in.z2z_fft);
    if (in.direct_f64) m.direct_pair = default_cost_model(2, true, in.es.w).direct_pair;
    double P[3], B[3];
    for (int d = 0; d < 3; ++d) {
        double lo = INFINITY, hi = -INFINITY;
        for (int64_t i = 0; i < in.n_pix; ++i) {
            lo = std::min(lo, in.pix[3 * i + d]);
            hi = std::max(hi, in.pix[3 * i + d]);
        }
        P[d] = hi - lo;
        lo = INFINITY;
        hi = -INFINITY;
        for (int64_t i = 0; i < in.n_vis; ++i) {
            lo = std::min(lo, in.uvw[3 * i + d]);
            hi = std::max(hi, in.uvw[3 * i + d]);
        }
        B[d] = hi - lo;
    }
    Evaluated best;
    double best_sigma = in.sigma;
    ESKernel best_es = in.es;
    // Problems whose whole direct evaluation (both directions) is modelled below the search
    // threshold are planned as one direct rectangle without a budget search: the search
    // (~1-3 us per point) would cost more than it could save over the plan's expected use.
    const bool tiny = 2.0 * m.direct_pair * (double)in.n_pix * (double)in.n_vis < in.search_threshold;
    if (in.budget > 0) {
        const double ratio =
            in.factor ? factored_ratio(in.factor, P, B, in.budget, in.sigma, in.es.w, in.elem_bytes) : 1.0;
        best = evaluate(in, m, in.budget, P, B, ratio);
    } else if (in.mode == HVOX_MODE_DIRECT || (tiny && in.mode == HVOX_MODE_AUTO && in.direct_threshold <= 0)) {
        PlanInputs direct = in;
        direct.mode = HVOX_MODE_DIRECT;
        best = evaluate(direct, m, 1e30, P, B);
    } else {
        // Upsampling search (sigma trades FFT cells, ~sigma^6, against kernel width) and
        // budget search: 256 KiB .. 8 GiB in factors of 8, capped by max_budget (the cost
        // model picks both). Candidates are evaluated on up to 4 threads; the choice is the
        // cheapest, the earliest candidate on ties, so it does not depend on the threading.
        struct Cand {
            double sigma, budget;
            ESKernel es;
        };
        std::vector<Cand> cands;
        std::vector<double> sigmas = in.sigma_auto ? std::vector<double>{2.0, 1.5, 1.25} : std::vector<double>{in.sigma};
        for (double sg : sigmas) {
            // an upsampling whose kernel would be wider than 16 cells is not a candidate
            if (in.sigma_auto && !in.fixed_w && es_width(in.eps_es, sg) > 16) continue;
            const ESKernel es = !in.sigma_auto ? in.es
                                : in.fixed_w   ? es_with_width(in.fixed_w, sg)
                                               : es_params(in.eps_es, sg);
            if (in.sigma_auto && in.prec == 1 && sg != sigmas.front()) {
                // FP32 grids: rounding errors near the band edge are divided twice by the
                // kernel transform (1/Psi before the FFT, 1/Phi after the interpolation),
                // so the error floor is about 2^-24 (Phi(0) / Phi(pi / sigma))^2. Smaller
                // sigma narrows the margin; keep a candidate only while the floor stays
                // within half of the 10 eps bound.
                const double tau[2] = {0.0, M_PI / sg};
                double ph[2];
                es_ft(es, tau, 2, ph);
                const double r = ph[0] / ph[1];
                if (std::ldexp(1.0, -24) * r * r > 5.0 * in.eps_es) continue;
            }
            for (double b = 256.0 * 1024.0; b <= 9.0e9; b *= 8.0) {
                if (in.max_budget > 0 && b > in.max_budget && b > 256.0 * 1024.0) break;
                cands.push_back({sg, b, es});
            }
        }
        if (cands.empty())
            fail(HVOX_EUNSUPPORTED, "no upsampling keeps the kernel within 16 cells at this tolerance");
        std::vector<Evaluated> evals(cands.size());
        const size_t width = std::max<size_t>(1, std::min<size_t>(4, std::thread::hardware_concurrency()));
        for (size_t c0 = 0; c0 < cands.size(); c0 += width) {
            std::vector<std::future<void>> jobs;
            for (size_t c = c0; c < std::min(cands.size(), c0 + width); ++c)
                jobs.push_back(std::async(std::launch::async, [&, c] {
                    PlanInputs cand = in;
                    cand.sigma = cands[c].sigma;
                    cand.es = cands[c].es;
                    const double ratio =
                        in.factor ? factored_ratio(in.factor, P, B, cands[c].budget, cand.sigma, cand.es.w,
                                                   in.elem_bytes)
                                  : 1.0;
                    evals[c] = evaluate(cand, m, cands[c].budget, P, B, ratio);
                }));
            for (auto &j : jobs) j.get();
            // keep only the best so far (bounds host memory on large point sets)
            for (size_t c = c0; c < std::min(cands.size(), c0 + width); ++c) {
                if (c == 0 || evals[c].cost < best.cost) {
                    best = std::move(evals[c]);
                    best_sigma = cands[c].sigma;
                    best_es = cands[c].es;
                }
                evals[c] = Evaluated();
            }
        }
        // Second pass: split the Heisenberg volume differently between pixel and baseline
        // boxes (the number of times each point is spread or gathered is the number of
        // chunks of the other set it meets). When the first pass found a NUFFT sub-problem
        // the ratios are tried at its upsampling and budget. When it found none (isotropic
        // boxes cut the sky into chunks too small to pay for a grid, as with a dense core
        // inside a long-baseline array) every budget is tried with ratios up to 64, so that
        // a core of short baselines can meet the whole sky in one box.
        // Both factored forms (one box spanning one of the sets, so that the other set's
        // points are spread once) are candidates at the chosen budget; a caller-fixed factor
        // skips this pass.
        if (best.cost > 0 && !in.factor) {
            const bool none = best.nufft_pairs.empty();
            std::vector<std::pair<double, double>> rb;  // (budget, ratio)
            for (int f : {1, 2}) {
                const double r = factored_ratio(f, P, B, best.budget, best_sigma, best_es.w, in.elem_bytes);
                if (r != 1.0) rb.push_back({best.budget, r});
            }
            if (!none) {
                for (double r : {0.25, 0.5, 2.0, 4.0, 8.0}) rb.push_back({best.budget, r});
            } else {
                for (double b = 256.0 * 1024.0; b <= 9.0e9; b *= 8.0) {
                    if (in.max_budget > 0 && b > in.max_budget && b > 256.0 * 1024.0) break;
                    for (double r : {4.0, 16.0, 64.0}) rb.push_back({b, r});
                    // the ratio at which one pixel box spans the whole sky (eta = P, with a
                    // hair of slack so that the extreme pixels do not start a second cell)
                    double eta[3], h[3];
                    const double t = box_dims(P, B, b, best_sigma, best_es.w, in.elem_bytes, eta, h);
                    if (t > 0.0 && t < 1.0) rb.push_back({b, 1.000001 / t});
                }
            }
            std::vector<Evaluated> rev(rb.size());
            PlanInputs cand = in;
            cand.sigma = best_sigma;
            cand.es = best_es;
            for (size_t c0 = 0; c0 < rb.size(); c0 += width) {
                std::vector<std::future<void>> jobs;
                for (size_t c = c0; c < std::min(rb.size(), c0 + width); ++c)
                    jobs.push_back(std::async(std::launch::async,
                                              [&, c] { rev[c] = evaluate(cand, m, rb[c].first, P, B, rb[c].second); }));
                for (auto &j : jobs) j.get();
                for (size_t c = c0; c < std::min(rb.size(), c0 + width); ++c) {
                    if (rev[c].cost < best.cost) best = std::move(rev[c]);
                    rev[c] = Evaluated();
                }
            }
        }
    }
    if (!std::isfinite(best.cost))
        fail(HVOX_EINVAL, "no feasible partition: a chunk budget must hold a grid of 2w cells per dimension "
                          "and give fewer than " + std::to_string((int64_t)kMaxCandidatePairs) +
                          " candidate sub-problems; set chunk_budget_bytes larger");
    r.box_ratio = best.ratio;
    r.sigma = best_sigma;
    r.es = best_es;
    r.t = best.t;
    r.budget = best.budget;
    for (int d = 0; d < 3; ++d) {
        r.h[d] = best.h[d];
        r.eta[d] = best.eta[d];
    }
    r.model_seconds = best.cost;
    r.pix_label = best.pl;
    r.vis_label = best.vl;
    r.n_pix_chunks = best.npc;
    r.n_vis_chunks = best.nvc;

    // Chunk order: chunks that take part in a NUFFT sub-problem first, then the rest,
    // each group in Algorithm 2 numbering. Points keep their original order inside a chunk.
    std::vector<char> pin(best.npc, 0), vin(best.nvc, 0);
    for (auto &pr : best.nufft_pairs) {
        pin[pr.first] = 1;
        vin[pr.second] = 1;
    }
    auto order_chunks = [](const std::vector<char> &flag) {
        std::vector<int64_t> ord;
        for (int64_t c = 0; c < (int64_t)flag.size(); ++c)
            if (flag[c]) ord.push_back(c);
        for (int64_t c = 0; c < (int64_t)flag.size(); ++c)
            if (!flag[c]) ord.push_back(c);
        return ord;
    };
    r.pix_chunk_label = order_chunks(pin);
    r.vis_chunk_label = order_chunks(vin);
    // Inside a chunk, points follow the Morton (Z-order) curve of their position in grid-cell
    // units: a pixel's grid coordinate along d is ~ sigma B_d r_d and a baseline's ~ sigma
    // P_d p_d, so dimension d is scaled by the other set's extent before quantising. Then
    // consecutive points are close on the grid (compact spreading tiles) even where one
    // dimension is thin, such as a sky cap's z.
    auto build_perm = [](const double *xyz, const std::vector<int64_t> &labels, int64_t nc,
                         const std::vector<int64_t> &ord, std::vector<int64_t> &perm, std::vector<int64_t> &start,
                         const double scale[3]) {
        const int64_t n = (int64_t)labels.size();
        std::vector<int64_t> rank(nc);
        for (int64_t k = 0; k < nc; ++k) rank[ord[k]] = k;
        std::vector<int64_t> cnt(nc + 1, 0);
        for (int64_t l : labels) cnt[rank[l] + 1]++;
        for (int64_t k = 0; k < nc; ++k) cnt[k + 1] += cnt[k];
        start = cnt;
        perm.assign(n, 0);
        std::vector<int64_t> pos(cnt.begin(), cnt.end() - 1);
        for (int64_t i = 0; i < n; ++i) perm[pos[rank[labels[i]]]++] = i;
        double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
        for (int64_t i = 0; i < n; ++i)
            for (int d = 0; d < 3; ++d) {
                lo[d] = std::min(lo[d], xyz[3 * i + d]);
                hi[d] = std::max(hi[d], xyz[3 * i + d]);
            }
        double span = 0.0;
        for (int d = 0; d < 3; ++d) span = std::max(span, (hi[d] - lo[d]) * scale[d]);
        std::vector<uint64_t> code(n);
        for (int64_t i = 0; i < n; ++i) {
            uint64_t c = 0;
            uint32_t q[3];
            for (int d = 0; d < 3; ++d) {
                double u = span > 0 ? (xyz[3 * i + d] - lo[d]) * scale[d] / span : 0.0;
                q[d] = (uint32_t)std::min(2097151.0, std::max(0.0, std::floor(u * 2097151.0)));
            }
            for (int bit = 20; bit >= 0; --bit)
                for (int d = 0; d < 3; ++d) c = (c << 1) | ((q[d] >> bit) & 1u);
            code[i] = c;
        }
        for (int64_t k = 0; k < nc; ++k)
            std::sort(perm.begin() + start[k], perm.begin() + start[k + 1], [&](int64_t a, int64_t b) {
                return code[a] != code[b] ? code[a] < code[b] : a < b;
            });
        return rank;
    };
    std::vector<int64_t> prank =
        build_perm(in.pix, best.pl, best.npc, r.pix_chunk_label, r.pix_perm, r.pix_chunk_start, B);
    std::vector<int64_t> vrank =
        build_perm(in.uvw, best.vl, best.nvc, r.vis_chunk_label, r.vis_perm, r.vis_chunk_start, P);

    // NUFFT blocks with their geometry.
    const double sigma = best_sigma;
    const int w = best_es.w;
    int64_t n_pin = 0, n_vin = 0;
    for (char f : pin) n_pin += f;
    for (char f : vin) n_vin += f;
    std::vector<std::vector<int64_t>> nufft_pix_of_v(n_vin);
    for (auto &pr : best.nufft_pairs) {
        int64_t i = pr.first, j = pr.second;
        NufftBlock b;
        b.pix_chunk = i;
        b.vis_chunk = j;
        int64_t pi = prank[i], vj = vrank[j];
        b.p0 = r.pix_chunk_start[pi];
        b.p1 = r.pix_chunk_start[pi + 1];
        b.v0 = r.vis_chunk_start[vj];
        b.v1 = r.vis_chunk_start[vj + 1];
        for (int d = 0; d < 3; ++d) {
            double plo = best.ps.lo[3 * i + d], phi = best.ps.hi[3 * i + d];
            double vlo = best.vs.lo[3 * j + d], vhi = best.vs.hi[3 * j + d];
            b.C[d] = 0.5 * (plo + phi);
            b.D[d] = 0.5 * (vlo + vhi);
            double X = 0.5 * (phi - plo), Bh = 0.5 * (vhi - vlo);
            grid_sizes(phi - plo, vhi - vlo, sigma, w, b.n1[d], b.n2[d]);
            if (X > 0.0)
                b.a[d] = (double)(b.n1[d] - w - 2) / (2.0 * X);
            else
                b.a[d] = 2.0 * sigma * Bh;
        }
        double pext[3], vext[3];
        for (int d = 0; d < 3; ++d) {
            pext[d] = best.ps.hi[3 * i + d] - best.ps.lo[3 * i + d];
            vext[d] = best.vs.hi[3 * j + d] - best.vs.lo[3 * j + d];
        }
        double cells = 0;
        b.cost = nufft_cost(m, best_es, sigma, b.p1 - b.p0, b.v1 - b.v0, pext, vext, &cells);
        double m1 = (double)(b.n1[0] * b.n1[1] * b.n1[2]), m2 = (double)(b.n2[0] * b.n2[1] * b.n2[2]);
        r.max_grid_bytes = std::max(r.max_grid_bytes, (double)in.elem_bytes * (m1 + m2));
        r.nufft_cells += cells;
        r.nufft_points += (double)(b.p1 - b.p0 + b.v1 - b.v0);
        r.nufft_pix_points += (double)(b.p1 - b.p0);
        r.nufft_vis_points += (double)(b.v1 - b.v0);
        r.spread_cells += m1;
        r.fft_work += m2 * std::log2(std::max(2.0, m2));
        r.blocks.push_back(b);
        nufft_pix_of_v[vj].push_back(pi);
    }
    // Largest-first ordering of NUFFT blocks (better overlap when several run at once).
    std::stable_sort(r.blocks.begin(), r.blocks.end(),
                     [](const NufftBlock &a, const NufftBlock &b) { return a.cost > b.cost; });

    // Direct rectangles.
    const int64_t p_split = r.pix_chunk_start[n_pin];
    const int64_t v_split = r.vis_chunk_start[n_vin];
    if (v_split < in.n_vis) r.rects.push_back({0, in.n_pix, v_split, in.n_vis});
    if (p_split < in.n_pix && v_split > 0) r.rects.push_back({p_split, in.n_pix, 0, v_split});
    for (int64_t vj = 0; vj < n_vin; ++vj) {
        std::vector<char> used(n_pin, 0);
        for (int64_t pi : nufft_pix_of_v[vj]) used[pi] = 1;
        int64_t v0 = r.vis_chunk_start[vj], v1 = r.vis_chunk_start[vj + 1];
        int64_t run = -1;
        for (int64_t pi = 0; pi <= n_pin; ++pi) {
            bool direct = pi < n_pin && !used[pi];
            if (direct && run < 0) run = pi;
            if (!direct && run >= 0) {
                r.rects.push_back({r.pix_chunk_start[run], r.pix_chunk_start[pi], v0, v1});
                run = -1;
            }
        }
    }
    for (auto &rc : r.rects) r.direct_pairs += (double)(rc.p1 - rc.p0) * (double)(rc.v1 - rc.v0);
    return r;
}

}  // namespace hvox
