// gbp_api.cu -- host side of libgbp: the C ABI declared in include/gbp.h.
//
// Owns the device buffers of one factor graph, builds the layout described
// in gbp_internal.h (factors sorted by landmark then keyframe, CSR lists),
// issues the kernels of gbp_kernels.cu on the caller's stream, replays the
// iteration loop as a CUDA graph, and converts chart means to world poses
// at the boundary.
#include "gbp_internal.h"
#include "gbp_mlp.cuh"
#include "../../include/gbp.h"

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <unordered_map>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <numeric>
#include <string>
#include <vector>

using namespace gbp;

static_assert(GBP_SPLIT_MSG_FLOATS == KREC + KJ, "split message record");
static_assert(GBP_SPLIT_KF_FLOATS == KBEL, "split keyframe record");

namespace {

constexpr int GRAPH_CHUNK = 8;   // iterations per captured CUDA graph

template <typename T>
cudaError_t dev_alloc(T** p, size_t n) {
    *p = nullptr;
    if (n == 0) n = 1;
    return cudaMalloc(reinterpret_cast<void**>(p), n * sizeof(T));
}

// Device buffers of a graph's layout, kept for reuse when a layout is
// replaced (a keyframe added): a released buffer goes back to the pool and
// the next layout takes the smallest one that fits.  With headroom > 1 a
// new buffer is allocated that much larger, so that the following layouts,
// each a little larger, find their buffers here instead of in cudaMalloc.
struct BufPool {
    std::unordered_map<void*, size_t> cap;       // pool buffers in use or free: their size
    std::vector<std::pair<size_t, void*>> spare; // released ones
    template <typename T>
    cudaError_t alloc(T** p, size_t n, double headroom) {
        const size_t bytes = std::max<size_t>(n, 1) * sizeof(T);
        size_t best = SIZE_MAX, at = 0;
        for (size_t i = 0; i < spare.size(); ++i)
            if (spare[i].first >= bytes && spare[i].first < best) {
                best = spare[i].first;
                at = i;
            }
        if (best != SIZE_MAX) {
            *p = static_cast<T*>(spare[at].second);
            spare.erase(spare.begin() + (long)at);
            return cudaSuccess;
        }
        const size_t want = std::max(bytes, size_t(double(bytes) * headroom));
        void* q = nullptr;
        cudaError_t e = cudaMalloc(&q, want);
        *p = static_cast<T*>(q);
        if (e == cudaSuccess) cap[q] = want;
        return e;
    }
    void put(void* p) {
        if (!p) return;
        auto it = cap.find(p);
        if (it == cap.end()) cudaFree(p);   // not from the pool
        else spare.emplace_back(it->second, p);
    }
    void clear() {
        for (auto& f : spare) {
            cap.erase(f.second);
            cudaFree(f.second);
        }
        spare.clear();
    }
};

template <typename R>
struct DevState {
    DevGraph<R> g{};
    // owned device pointers (non-const views of g)
    R* z = nullptr;
    int32_t* fk = nullptr;
    int32_t* fm = nullptr;
    double* kf_R = nullptr;
    double* kf_c = nullptr;
    double* lm_ref = nullptr;
    R* kf_Rr = nullptr;
    R* f_dlc = nullptr;
    int32_t* kf_off = nullptr;
    int32_t* kf_list = nullptr;
    int32_t* kpos = nullptr;
    int32_t* lm_off = nullptr;
    int32_t* tile_start = nullptr;
    int32_t* big_lm = nullptr;
    int32_t* deferred = nullptr;
    int32_t* orphan = nullptr;
    int32_t* kf_birth = nullptr;
    int32_t* lm_birth = nullptr;
    R* kf_D = nullptr;
    R* kf_A = nullptr;
    R* lm_D = nullptr;
    R* uv_ref = nullptr;
    R* x0 = nullptr;
    int32_t* tlin = nullptr;
    R* mk = nullptr;
    R* mk2 = nullptr;
    R* kj = nullptr;
    R* kjs = nullptr;
    R* lin = nullptr;
    R* ml = nullptr;
    R* mlx = nullptr;
    R* kf_bel = nullptr;
    R* lm_bel = nullptr;
    R* prior_s = nullptr;      // prior scale table, prior_anneal_iters + 1 entries
    float* hist = nullptr;     // learned damping: HIST x n_f message-change history
    R* eta_inf = nullptr;      // record schedule: 9 x n_f reference messages (gbp_capture_messages)

    // every buffer freed, or (pool given) handed back to the pool
    void release(BufPool* pool = nullptr) {
        void* ptrs[] = {z, fk, fm, kf_R, kf_c, lm_ref, kf_Rr, f_dlc, kf_off, kf_list, kpos, lm_off, tile_start, big_lm, deferred, orphan, kf_birth, lm_birth, kf_D, kf_A, lm_D,
                        uv_ref, x0, tlin, mk, mk2, kj, kjs, lin, ml, mlx, kf_bel, lm_bel, prior_s, hist, eta_inf};
        for (void* p : ptrs)
            if (p) {
                if (pool) pool->put(p);
                else cudaFree(p);
            }
        *this = DevState<R>();
    }
};

// Exp of so(3) in double for the boundary conversion (Rodrigues' formula).
void so3_exp_host(const double w[3], double E[9]) {
    double th2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
    double a, b;
    if (th2 < 1e-12) {
        a = 1.0 - th2 / 6.0;
        b = 0.5 - th2 / 24.0;
    } else {
        double th = std::sqrt(th2);
        double sh = std::sin(0.5 * th);
        a = std::sin(th) / th;
        b = 2.0 * sh * sh / th2;
    }
    double W[9] = {0, -w[2], w[1], w[2], 0, -w[0], -w[1], w[0], 0};
    double W2[9] = {w[0] * w[0] - th2, w[0] * w[1], w[0] * w[2], w[1] * w[0], w[1] * w[1] - th2, w[1] * w[2],
                    w[2] * w[0], w[2] * w[1], w[2] * w[2] - th2};
    for (int i = 0; i < 9; ++i) E[i] = a * W[i] + b * W2[i];
    E[0] += 1.0; E[4] += 1.0; E[8] += 1.0;
}

// The keyframe belief record of a prior-only belief (diagonal p): its
// Cholesky factor (1/sqrt(p_i) on the diagonal), mean 0, trace, Lambda.
template <typename R>
void kf_prior_record_host(const R* p, R* out) {
    std::fill(out, out + KBEL, R(0));
    R tr = R(0);
    for (int i = 0; i < 6; ++i) {
        out[KB_L + i * (i + 1) / 2 + i] = R(1.0 / std::sqrt(double(p[i])));
        out[KB_LAM + i * (i + 1) / 2 + i] = p[i];
        tr += p[i];
    }
    out[KB_TR] = tr;
}

}  // namespace

struct gbp_graph {
    std::string err;
    BufPool pool;                       // buffers of replaced layouts, for the next one
    double headroom = 1.0;              // > 1 once keyframes are added: layouts grow
    cudaStream_t stream = nullptr;      // caller's stream (may be the legacy default)
    cudaStream_t capture = nullptr;     // private stream used only to record CUDA graphs
    gbp_intrinsics intr{};
    gbp_params prm{};
    int n_kf = 0, n_lm = 0, n_f = 0;
    // host copy of the problem (internal factor order)
    std::vector<double> kf_R, kf_c, lm_ref;     // references (chart origins)
    std::vector<int32_t> fk, fm, obs_index;     // obs_index[f] = caller's observation index
    std::vector<double> z;
    std::vector<uint8_t> anchored;
    std::vector<int32_t> kf_birth, lm_birth;    // iteration each variable was added at (prior anneal start)
    std::vector<int32_t> prob_kf0, prob_lm0;    // problem table (n_problems + 1 entries, last = totals)
    std::vector<int32_t> prob_f0;               // first internal factor of each problem (+ total)
    int32_t* d_prob_f0 = nullptr;               // device copy for the per-problem metrics
    std::vector<double> uv_ref;                 // reference projections (internal order) or empty
    // device
    int storage = 0;                            // 0: float, 1: double
    DevState<float> sf;
    DevState<double> sd;
    int32_t* ctl = nullptr;
    double* partials = nullptr;
    double* met = nullptr;
    int n_partials = 0;
    int32_t* h_ctl = nullptr;                   // pinned mirror of ctl
    double* h_met = nullptr;                    // pinned mirror of met
    cudaGraphExec_t exec = nullptr;
    cudaGraphExec_t wexec = nullptr;            // device convergence loop (conditional WHILE node)
    int wexec_every = 0;                        // its check_every
    bool wexec_failed = false;                  // not available for this layout: the host checks
    bool built = false;
    int tuned_mode = 0;                         // autotuner's choice (1 or 2), 0 = not tuned
    int tuned_fshape = -1, tuned_pshape = -1;   // its launch shapes, -1 = not tuned
    // one graph split across ranks (gbp_set_partition): the keyframes and
    // landmarks whose beliefs this graph forms; lm1 < 0 = not split
    int part_kf0 = 0, part_kf1 = -1, part_lm0 = 0, part_lm1 = -1;
    std::vector<int32_t> f_of_obs;              // internal factor of each caller observation
    gbp_tuning tuning{};                        // candidates of the last gbp_autotune
    int last_mode = 0;                          // launch mode of the last gbp_iterate()
    int64_t launches = 0;                       // kernels launched (graph replays count their kernels)
    bool pdl = true;                            // programmatic dependent launch between the per-phase kernels
    // learned damping: the graph's own copy of a network's packed weights
    uint32_t* mlp_frag = nullptr;
    float* mlp_bias = nullptr;
    bool has_model = false;
};

namespace {

gbp_status fail(gbp_graph* g, gbp_status s, const std::string& msg) {
    if (g) g->err = msg;
    return s;
}

gbp_status cuda_fail(gbp_graph* g, cudaError_t e, const char* where) {
    std::string m = std::string(where) + ": " + cudaGetErrorString(e);
    return fail(g, GBP_ECUDA, m);
}

#define CK(expr)                                                   \
    do {                                                           \
        cudaError_t e_ = (expr);                                   \
        if (e_ != cudaSuccess) return cuda_fail(g, e_, #expr);     \
    } while (0)

template <typename R>
DevState<R>& state(gbp_graph* g);

template <typename R>
KParams<R> make_kparams(gbp_graph* g) {
    const gbp_params& p = g->prm;
    KParams<R> k{};
    k.fx = R(g->intr.fx);
    k.fy = R(g->intr.fy);
    k.cx = R(g->intr.cx);
    k.cy = R(g->intr.cy);
    k.inv_sigma2 = R(1.0 / (double(p.sigma_px) * double(p.sigma_px)));
    k.inv_sigma = R(1.0 / double(p.sigma_px));
    k.huber_n = R(p.huber_nsigma);
    k.damping = R(p.damping);
    k.z_min = R(p.z_min);
    k.relin_beta = R(p.relin_beta);
    k.anchor_scale = R(p.anchor_scale);
    k.pivot_ratio = R(p.fp64_pivot_ratio);
    // a keyframe cavity keeping less than 1/1000 of its belief's precision
    // volume amplifies FP32 rounding by up to 1000x: formed again in FP64
    // (every one of them with fp64_pivot_ratio >= 1)
    k.cav_ratio = R(std::max(1e-3, double(p.fp64_pivot_ratio)));
    k.prior_s = state<R>(g).prior_s;
    k.prior_T = std::max(p.prior_anneal_iters, 0);
    k.relin_interval = p.relin_interval;
    k.damp_hold = std::max(p.undamped_iters, 1);
    k.linear = p.linear;
    k.fallback = p.precision_mode == 0 ? 1 : 0;
    k.exact_cavity = p.fp64_exact_cavity;
    k.mlp_frag = g->mlp_frag;
    k.mlp_bias = g->mlp_bias;
    return k;
}

// Launch shapes in use: the parameter if set, else the autotuner's choice,
// else by size (large graphs -- a warp per belief item -- take the deferring
// kernel at >= 4 blocks per SM, which measured fastest there).
bool tunable(const gbp_graph* g) { return g->storage == 0 && g->prm.damping_mode == 0; }
int factor_shape(const gbp_graph* g) {
    if (!tunable(g)) return 0;
    if (g->prm.factor_shape >= 0) return g->prm.factor_shape;
    if (g->tuned_fshape >= 0) return g->tuned_fshape;
    return g->sf.g.b_warps == 1 ? 4 : 0;
}
// The persistent kernel runs in one shape, with no register budget: under
// a budget (>= 3 or >= 4 blocks per SM) it compiled to different rounding
// from the per-phase kernels (measured), and it is the slower launch mode
// at every size measured, so budgets are not offered.
int n_persistent_shapes(const gbp_graph*) { return N_PERSISTENT_SHAPES; }
int persistent_shape(const gbp_graph*) { return 0; }

void destroy_exec(gbp_graph* g) {
    if (g->exec) {
        cudaGraphExecDestroy(g->exec);
        g->exec = nullptr;
    }
    if (g->wexec) {
        cudaGraphExecDestroy(g->wexec);
        g->wexec = nullptr;
    }
    g->wexec_failed = false;
}

template <>
DevState<float>& state<float>(gbp_graph* g) { return g->sf; }
template <>
DevState<double>& state<double>(gbp_graph* g) { return g->sd; }

// Sec. 8: prior scale s(t) = prior_final_scale^(min(t, T) / T), tabulated
// for t = 0..T (T = prior_anneal_iters; T = 0 means the final scale
// throughout) and uploaded for the kernels.
template <typename R>
gbp_status upload_prior_table(gbp_graph* g) {
    DevState<R>& s = state<R>(g);
    const int T = std::max(g->prm.prior_anneal_iters, 0);
    std::vector<R> tab(T + 1);
    for (int t = 0; t <= T; ++t)
        tab[t] = T == 0 ? R(g->prm.prior_final_scale)
                        : R(std::pow(double(g->prm.prior_final_scale), double(t) / double(T)));
    if (s.prior_s) cudaFree(s.prior_s);
    s.prior_s = nullptr;
    CK(dev_alloc(&s.prior_s, tab.size()));
    CK(cudaMemcpyAsync(s.prior_s, tab.data(), sizeof(R) * tab.size(), cudaMemcpyHostToDevice, g->stream));
    CK(cudaStreamSynchronize(g->stream));
    return GBP_OK;
}

// Upload the problem into freshly allocated device buffers of type R and
// generate the priors; leaves the dynamic state uninitialised.
template <typename R>
// x0_init: linearisation points for the prior pass (host), or rs: gathered
// on the device from a previous layout (a keyframe was added), else zero.
gbp_status build_device(gbp_graph* g, const std::vector<R>* x0_init = nullptr, const RelayoutSrc<R>* rs = nullptr) {
    DevState<R>& s = state<R>(g);
    s.release(&g->pool);
    const int nk = g->n_kf, nl = g->n_lm, nf = g->n_f;
    // CSR lists
    std::vector<int32_t> kf_off(nk + 1, 0), lm_off(nl + 1, 0), kf_list(nf);
    for (int f = 0; f < nf; ++f) {
        kf_off[g->fk[f] + 1]++;
        lm_off[g->fm[f] + 1]++;
    }
    for (int v = 0; v < nk; ++v) kf_off[v + 1] += kf_off[v];
    for (int v = 0; v < nl; ++v) lm_off[v + 1] += lm_off[v];
    std::vector<int32_t> kpos(nf);
    {
        std::vector<int32_t> fill(kf_off.begin(), kf_off.end() - 1);
        for (int f = 0; f < nf; ++f) {
            kpos[f] = fill[g->fk[f]]++;
            kf_list[kpos[f]] = f;
        }
    }
    // warp tiles: consecutive whole landmarks, at most 32 factors per tile;
    // a landmark with more factors gets tiles of its own and its belief is
    // formed in the belief phase.  Variables without factors are orphans.
    std::vector<int32_t> tiles(1, 0), orphan, big;
    for (int v = 0; v < nk; ++v)
        if (kf_off[v + 1] == kf_off[v]) orphan.push_back(v);
    {
        // a tile never spans two problems of a batch, nor the landmark range
        // of a partition
        std::vector<int32_t> breaks(g->prob_lm0.begin() + 1, g->prob_lm0.end() - 1);
        if (g->part_lm1 >= 0) {
            breaks.push_back(g->part_lm0);
            breaks.push_back(g->part_lm1);
        }
        std::sort(breaks.begin(), breaks.end());
        int cur = 0;
        size_t next_brk = 0;
        for (int m = 0; m < nl; ++m) {
            const int lo = lm_off[m], hi = lm_off[m + 1], d = hi - lo;
            while (next_brk < breaks.size() && breaks[next_brk] <= m) {
                if (breaks[next_brk] == m && cur > 0) {
                    tiles.push_back(lo);
                    cur = 0;
                }
                ++next_brk;
            }
            if (d == 0) {
                orphan.push_back(nk + m);
                continue;
            }
            if (d > 32) {
                if (cur > 0) {
                    tiles.push_back(lo);
                    cur = 0;
                }
                for (int x = lo + 32; x < hi; x += 32) tiles.push_back(x);
                tiles.push_back(hi);
                big.push_back(m);
                continue;
            }
            if (cur + d > 32) {
                tiles.push_back(lo);
                cur = 0;
            }
            cur += d;
        }
        if (cur > 0) tiles.push_back(nf);
    }
    const int n_tiles = (int)tiles.size() - 1;
    std::vector<R> zr(2 * (size_t)nf), anc(6 * (size_t)nk, R(0));
    for (size_t i = 0; i < zr.size(); ++i) zr[i] = R(g->z[i]);
    // the linearisation's references in R: the rotation rounded, and each
    // factor's point-minus-centre difference taken in double, then rounded
    std::vector<R> rr(9 * (size_t)nk), dlc(3 * (size_t)nf);
    for (size_t i = 0; i < rr.size(); ++i) rr[i] = R(g->kf_R[i]);
    for (int f = 0; f < nf; ++f)
        for (int j = 0; j < 3; ++j)
            dlc[(size_t)j * nf + f] = R(g->lm_ref[3 * (size_t)g->fm[f] + j] - g->kf_c[3 * (size_t)g->fk[f] + j]);
    for (int v = 0; v < nk; ++v)
        if (g->anchored[v])
            for (int i = 0; i < 6; ++i) anc[6 * v + i] = R(1);   // scaled by D after the prior pass

    CK(g->pool.alloc(&s.z, 2 * (size_t)nf, g->headroom));
    CK(g->pool.alloc(&s.fk, nf, g->headroom));
    CK(g->pool.alloc(&s.fm, nf, g->headroom));
    CK(g->pool.alloc(&s.kf_R, 9 * (size_t)nk, g->headroom));
    CK(g->pool.alloc(&s.kf_c, 3 * (size_t)nk, g->headroom));
    CK(g->pool.alloc(&s.lm_ref, 3 * (size_t)nl, g->headroom));
    CK(g->pool.alloc(&s.kf_Rr, 9 * (size_t)nk, g->headroom));
    CK(g->pool.alloc(&s.f_dlc, 3 * (size_t)nf, g->headroom));
    CK(g->pool.alloc(&s.kf_off, nk + 1, g->headroom));
    CK(g->pool.alloc(&s.kf_list, nf, g->headroom));
    CK(g->pool.alloc(&s.kpos, nf, g->headroom));
    CK(g->pool.alloc(&s.lm_off, nl + 1, g->headroom));
    CK(g->pool.alloc(&s.tile_start, tiles.size(), g->headroom));
    CK(g->pool.alloc(&s.big_lm, big.size(), g->headroom));
    CK(g->pool.alloc(&s.deferred, (size_t)n_tiles, g->headroom));
    CK(g->pool.alloc(&s.orphan, orphan.size(), g->headroom));
    CK(g->pool.alloc(&s.kf_birth, nk, g->headroom));
    CK(g->pool.alloc(&s.lm_birth, nl, g->headroom));
    CK(g->pool.alloc(&s.kf_D, 6 * (size_t)nk, g->headroom));
    CK(g->pool.alloc(&s.kf_A, 6 * (size_t)nk, g->headroom));
    CK(g->pool.alloc(&s.lm_D, 3 * (size_t)nl, g->headroom));
    CK(g->pool.alloc(&s.x0, 9 * (size_t)nf, g->headroom));
    CK(g->pool.alloc(&s.tlin, nf, g->headroom));
    CK(g->pool.alloc(&s.mk, (size_t)KREC * nf, g->headroom));
    CK(g->pool.alloc(&s.mk2, (size_t)KREC * nf, g->headroom));
    CK(g->pool.alloc(&s.kj, (size_t)KJ * nf, g->headroom));
    CK(g->pool.alloc(&s.kjs, (size_t)KJ * nf, g->headroom));
    CK(g->pool.alloc(&s.lin, (size_t)NLIN * nf, g->headroom));
    CK(g->pool.alloc(&s.ml, (size_t)NML * nf, g->headroom));
    CK(g->pool.alloc(&s.mlx, 9 * (size_t)nf, g->headroom));
    CK(g->pool.alloc(&s.kf_bel, (size_t)KBEL * nk, g->headroom));
    CK(g->pool.alloc(&s.lm_bel, (size_t)LBEL * nl, g->headroom));
    CK(g->pool.alloc(&s.hist, HIST * (size_t)std::max(nf, 1), g->headroom));
    cudaStream_t st = g->stream;
    CK(cudaMemcpyAsync(s.z, zr.data(), sizeof(R) * zr.size(), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(s.fk, g->fk.data(), sizeof(int32_t) * nf, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(s.fm, g->fm.data(), sizeof(int32_t) * nf, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(s.kf_R, g->kf_R.data(), sizeof(double) * 9 * nk, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(s.kf_c, g->kf_c.data(), sizeof(double) * 3 * nk, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(s.lm_ref, g->lm_ref.data(), sizeof(double) * 3 * nl, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(s.kf_Rr, rr.data(), sizeof(R) * rr.size(), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(s.f_dlc, dlc.data(), sizeof(R) * dlc.size(), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(s.kf_off, kf_off.data(), sizeof(int32_t) * (nk + 1), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(s.kf_list, kf_list.data(), sizeof(int32_t) * nf, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(s.kpos, kpos.data(), sizeof(int32_t) * nf, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(s.lm_off, lm_off.data(), sizeof(int32_t) * (nl + 1), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(s.tile_start, tiles.data(), sizeof(int32_t) * tiles.size(), cudaMemcpyHostToDevice, st));
    if (!orphan.empty())
        CK(cudaMemcpyAsync(s.orphan, orphan.data(), sizeof(int32_t) * orphan.size(), cudaMemcpyHostToDevice, st));
    if (!big.empty())
        CK(cudaMemcpyAsync(s.big_lm, big.data(), sizeof(int32_t) * big.size(), cudaMemcpyHostToDevice, st));
    if (nk) CK(cudaMemcpyAsync(s.kf_birth, g->kf_birth.data(), sizeof(int32_t) * nk, cudaMemcpyHostToDevice, st));
    if (nl) CK(cudaMemcpyAsync(s.lm_birth, g->lm_birth.data(), sizeof(int32_t) * nl, cudaMemcpyHostToDevice, st));
    // linearisation points (the references at creation) for the prior pass
    if (x0_init && nf)
        CK(cudaMemcpyAsync(s.x0, x0_init->data(), sizeof(R) * 9 * (size_t)nf, cudaMemcpyHostToDevice, st));
    else if (nf && !rs)
        CK(cudaMemsetAsync(s.x0, 0, sizeof(R) * 9 * (size_t)nf, st));

    DevGraph<R>& d = s.g;
    d.n_kf = nk;
    d.n_lm = nl;
    d.n_f = nf;
    d.z = s.z;
    d.fk = s.fk;
    d.fm = s.fm;
    d.kf_R = s.kf_R;
    d.kf_c = s.kf_c;
    d.lm_ref = s.lm_ref;
    d.kf_Rr = s.kf_Rr;
    d.f_dlc = s.f_dlc;
    d.kf_off = s.kf_off;
    d.kf_list = s.kf_list;
    d.kpos = s.kpos;
    d.lm_off = s.lm_off;
    d.tile_start = s.tile_start;
    d.big_lm = s.big_lm;
    d.deferred = s.deferred;
    d.orphan = s.orphan;
    d.kf_birth = s.kf_birth;
    d.lm_birth = s.lm_birth;
    d.n_tiles = n_tiles;
    d.n_big = (int32_t)big.size();
    d.n_orphan = (int32_t)orphan.size();
    d.tile_off = 0;
    d.kf_item_off = 0;
    d.kf_item_n = nk;
    d.big_item_off = 0;
    d.big_item_n = d.n_big;
    if (g->part_lm1 >= 0) {
        // this rank's tiles: those of its landmarks (contiguous, tiles break
        // at the range's ends); its split landmarks likewise
        int t0 = 0, t1 = 0;
        for (int t = 0; t < n_tiles; ++t) {
            const int lm = g->fm[tiles[t]];
            if (lm < g->part_lm0) t0 = t + 1;
            if (lm < g->part_lm1) t1 = t + 1;
        }
        int b0 = 0, b1 = 0;
        for (size_t i = 0; i < big.size(); ++i) {
            if (big[i] < g->part_lm0) b0 = (int)i + 1;
            if (big[i] < g->part_lm1) b1 = (int)i + 1;
        }
        d.tile_off = t0;
        d.n_tiles = t1 - t0;
        d.kf_item_off = g->part_kf0;
        d.kf_item_n = g->part_kf1 - g->part_kf0;
        d.big_item_off = b0;
        d.big_item_n = b1 - b0;
    }
    {
        // a block per belief item while a warp per item would leave SMs
        // idle (at most one block of FACTOR_BLOCK / 32 items per SM), else
        // a warp per item, so that the single-thread solves of many
        // keyframes run side by side (decided on the whole graph, so that
        // every part of a split graph sums as the whole graph would)
        int dev = 0, sms = 0;
        CK(cudaGetDevice(&dev));
        CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        d.b_warps = (nk + (int)big.size()) <= sms * (FACTOR_BLOCK / 32) ? FACTOR_BLOCK / 32 : 1;
    }
    d.kf_D = s.kf_D;
    d.kf_A = s.kf_A;
    d.lm_D = s.lm_D;
    d.uv_ref = nullptr;
    d.x0 = s.x0;
    d.tlin = s.tlin;
    d.mk = s.mk;
    d.mk2 = s.mk2;
    d.mk_redirect = nullptr;
    d.kj = s.kj;
    d.kjs = s.kjs;
    d.lin = s.lin;
    d.ml = s.ml;
    d.ml_out = s.ml;
    d.mlx = s.mlx;
    d.kf_bel = s.kf_bel;
    d.lm_bel = s.lm_bel;
    d.kf_bel_out = s.kf_bel;
    d.lm_bel_out = s.lm_bel;
    d.hist = s.hist;
    d.eta_inf = nullptr;
    d.rec_X = nullptr;
    d.rec_T = nullptr;
    d.ctl = g->ctl;
    if (rs && nf) CK(launch_relayout<R>(d, *rs, 0, st));

    // priors: per-factor diagonal information at the reference (temporary
    // buffers reuse the message storage, which is cleared afterwards)
    {
        gbp_status pst = upload_prior_table<R>(g);
        if (pst != GBP_OK) return pst;
    }
    KParams<R> kp = make_kparams<R>(g);
    CK(launch_prior<R>(d, kp, s.mk, s.ml, s.kf_D, s.lm_D, st));
    // anchor diagonal = D on anchored keyframes
    {
        std::vector<R> D(6 * (size_t)nk);
        CK(cudaMemcpyAsync(D.data(), s.kf_D, sizeof(R) * D.size(), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        for (size_t i = 0; i < D.size(); ++i) anc[i] *= D[i];
        CK(cudaMemcpyAsync(s.kf_A, anc.data(), sizeof(R) * anc.size(), cudaMemcpyHostToDevice, st));
    }
    if (!g->uv_ref.empty()) {
        std::vector<R> u(g->uv_ref.size());
        for (size_t i = 0; i < u.size(); ++i) u[i] = R(g->uv_ref[i]);
        CK(g->pool.alloc(&s.uv_ref, u.size(), g->headroom));
        CK(cudaMemcpyAsync(s.uv_ref, u.data(), sizeof(R) * u.size(), cudaMemcpyHostToDevice, st));
        d.uv_ref = s.uv_ref;
    }
    CK(cudaStreamSynchronize(st));
    return GBP_OK;
}

// Iteration 0: factors linearised at their references, messages zero,
// beliefs = prior(0).
template <typename R>
gbp_status reset_state(gbp_graph* g) {
    DevState<R>& s = state<R>(g);
    cudaStream_t st = g->stream;
    const size_t nf = g->n_f;
    CK(cudaMemsetAsync(s.x0, 0, sizeof(R) * 9 * nf, st));
    CK(cudaMemsetAsync(s.tlin, 0, sizeof(int32_t) * nf, st));
    CK(cudaMemsetAsync(s.mk, 0, sizeof(R) * KREC * nf, st));
    CK(cudaMemsetAsync(s.mk2, 0, sizeof(R) * KREC * nf, st));
    CK(cudaMemsetAsync(s.kj, 0, sizeof(R) * KJ * nf, st));
    CK(cudaMemsetAsync(s.kjs, 0, sizeof(R) * KJ * nf, st));
    CK(cudaMemsetAsync(s.lin, 0, sizeof(R) * NLIN * nf, st));
    CK(cudaMemsetAsync(s.ml, 0, sizeof(R) * NML * nf, st));
    CK(cudaMemsetAsync(s.mlx, 0, sizeof(R) * 9 * nf, st));
    CK(cudaMemsetAsync(s.kf_bel, 0, sizeof(R) * KBEL * g->n_kf, st));
    CK(cudaMemsetAsync(s.lm_bel, 0, sizeof(R) * LBEL * g->n_lm, st));
    CK(cudaMemsetAsync(s.hist, 0, sizeof(float) * HIST * nf, st));
    int32_t c0[CTL_N] = {0};
    CK(cudaMemcpyAsync(g->ctl, c0, sizeof(c0), cudaMemcpyHostToDevice, st));
    CK(launch_init<R>(s.g, make_kparams<R>(g), st));
    g->launches += 1;
    return GBP_OK;
}

gbp_status ensure_built(gbp_graph* g) {
    int want = g->prm.precision_mode == 2 ? 1 : 0;
    if (g->built && want == g->storage) return GBP_OK;
    destroy_exec(g);
    g->sf.release(&g->pool);
    g->sd.release(&g->pool);
    g->storage = want;
    gbp_status st = want ? build_device<double>(g) : build_device<float>(g);
    if (st != GBP_OK) return st;
    st = want ? reset_state<double>(g) : reset_state<float>(g);
    if (st != GBP_OK) return st;
    g->built = true;
    return GBP_OK;
}

template <typename R>
cudaError_t enqueue_iterations(gbp_graph* g, int n, cudaStream_t st) {
    const DevGraph<R>& d = state<R>(g).g;
    KParams<R> kp = make_kparams<R>(g);
    for (int i = 0; i < n; ++i) {
        cudaError_t e = launch_factor<R>(d, kp, st, g->prm.damping_mode, g->pdl, factor_shape(g));
        if (e != cudaSuccess) return e;
        e = launch_belief<R>(d, kp, st, g->pdl);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Record GRAPH_CHUNK iterations as a CUDA graph.  With programmatic
// dependent launch between the kernels if the capture accepts it, else
// (and from then on) with plain stream order.
gbp_status ensure_exec(gbp_graph* g) {
    if (g->exec) return GBP_OK;
    for (int attempt = 0; attempt < 2; ++attempt) {
        cudaGraph_t graph = nullptr;
        CK(cudaStreamBeginCapture(g->capture, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = g->storage ? enqueue_iterations<double>(g, GRAPH_CHUNK, g->capture)
                                   : enqueue_iterations<float>(g, GRAPH_CHUNK, g->capture);
        cudaError_t e2 = cudaStreamEndCapture(g->capture, &graph);
        if (e == cudaSuccess && e2 == cudaSuccess) {
            e = cudaGraphInstantiate(&g->exec, graph, 0);
            cudaGraphDestroy(graph);
            if (e == cudaSuccess) return GBP_OK;
            g->exec = nullptr;
        } else if (graph) {
            cudaGraphDestroy(graph);
        }
        if (!g->pdl) {
            if (e == cudaSuccess) e = e2;
            return cuda_fail(g, e, "capture");
        }
        cudaGetLastError();
        g->pdl = false;
    }
    return fail(g, GBP_ECUDA, "capture");
}

// Device convergence loop.  With conv_tol > 0 the per-phase launches are
// checked every check_every iterations; instead of a host round trip per
// check (a device-to-host copy and a stream synchronisation, during which
// the GPU idles), one graph launch runs the check blocks in a conditional
// WHILE node: its body is check_every iterations followed by a one-thread
// kernel that makes the host loop's test -- the largest mean change of the
// last iteration below conv_tol, no error raised -- and sets the loop's
// condition.  The kernels, their order and the check points are the host
// loop's, so the results and the iteration count are the same.  Two control
// slots past the kernels' own (the Ctl enum ends at CTL_RESUMS) carry the
// loop's state.
constexpr int CTL_WL_LEFT = 18;     // check blocks the loop may still run
constexpr int CTL_WL_TOL = 19;      // conv_tol, float bits
static_assert(CTL_WL_LEFT > CTL_RESUMS && CTL_WL_TOL < CTL_N, "control slots of the device loop");
constexpr int WHILE_MAX_BODY = 64;  // longest check block recorded in the loop body

__global__ void while_setup_kernel(int32_t* ctl, int32_t blocks, int32_t tol_bits) {
    ctl[CTL_WL_LEFT] = blocks;
    ctl[CTL_WL_TOL] = tol_bits;
}

__global__ void while_check_kernel(int32_t* ctl, cudaGraphConditionalHandle h) {
    const int left = ctl[CTL_WL_LEFT] - 1;
    ctl[CTL_WL_LEFT] = left;
    const int t = ctl[CTL_ITER];
    const float dmu = t > 0 ? __int_as_float(ctl[((t - 1) & 1) ? CTL_DMU_ACC1 : CTL_DMU_ACC]) : 0.0f;
    const float tol = __int_as_float(ctl[CTL_WL_TOL]);
    const bool go = left > 0 && !(dmu < tol) && ctl[CTL_ERR] == 0;
    cudaGraphSetConditional(h, go ? 1u : 0u);
}

// Records the loop (after ensure_exec, which settles g->pdl).  Where the
// driver does not take it (or check_every exceeds WHILE_MAX_BODY), the host
// loop checks instead.
gbp_status ensure_wexec(gbp_graph* g) {
    const int every = g->prm.check_every;
    if (g->wexec && g->wexec_every == every) return GBP_OK;
    if (g->wexec) {
        cudaGraphExecDestroy(g->wexec);
        g->wexec = nullptr;
    }
    if (g->wexec_failed || every > WHILE_MAX_BODY) return GBP_OK;
    cudaGraph_t graph = nullptr;
    cudaGraphConditionalHandle h = 0;
    cudaError_t e = cudaGraphCreate(&graph, 0);
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault);
    cudaGraphNodeParams cp = {};
    cudaGraphNode_t node = nullptr;
    if (e == cudaSuccess) {
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp);
    }
    if (e == cudaSuccess) {
        e = cudaStreamBeginCaptureToGraph(g->capture, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                          cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t e1 = g->storage ? enqueue_iterations<double>(g, every, g->capture)
                                        : enqueue_iterations<float>(g, every, g->capture);
            if (e1 == cudaSuccess) {
                while_check_kernel<<<1, 1, 0, g->capture>>>(g->ctl, h);
                e1 = cudaGetLastError();
            }
            cudaGraph_t body = nullptr;
            const cudaError_t e2 = cudaStreamEndCapture(g->capture, &body);
            e = e1 != cudaSuccess ? e1 : e2;
        }
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&g->wexec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        g->wexec = nullptr;
        g->wexec_failed = true;
        (void)cudaGetLastError();   // the host loop takes over; nothing of this is the caller's error
        return GBP_OK;
    }
    g->wexec_every = every;
    return GBP_OK;
}

// max |dmu| of the last completed iteration, from the mirrored control
// block: both launch modes leave it in the parity slot of that iteration.
float last_dmu(const gbp_graph* g) {
    const int t = g->h_ctl[CTL_ITER];
    if (t <= 0) return 0.0f;
    float v;
    std::memcpy(&v, &g->h_ctl[((t - 1) & 1) ? CTL_DMU_ACC1 : CTL_DMU_ACC], sizeof v);
    return v;
}

gbp_status read_ctl(gbp_graph* g) {
    CK(cudaMemcpyAsync(g->h_ctl, g->ctl, sizeof(int32_t) * CTL_N, cudaMemcpyDeviceToHost, g->stream));
    CK(cudaStreamSynchronize(g->stream));
    if (g->h_ctl[CTL_ERR] == 2)
        return fail(g, GBP_ETIMEOUT, "grid barrier wait exceeded its limit (blocks not co-resident?)");
    if (g->h_ctl[CTL_ERR]) {
        int w = g->h_ctl[CTL_ERR_WHERE];
        char buf[160];
        snprintf(buf, sizeof buf, "variable %d: belief not positive definite or mean not finite", w);
        return fail(g, GBP_EDIVERGED, buf);
    }
    return GBP_OK;
}

bool finite_all(const double* p, size_t n) {
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(p[i])) return false;
    return true;
}

gbp_status check_params(const gbp_params* p, std::string& why) {
    if (!(p->sigma_px > 0.0f) || !std::isfinite(p->sigma_px)) { why = "sigma_px must be > 0"; return GBP_EINVAL; }
    if (!(p->damping >= 0.0f && p->damping < 1.0f)) { why = "damping must be in [0, 1)"; return GBP_EINVAL; }
    if (!std::isfinite(p->huber_nsigma)) { why = "huber_nsigma must be finite"; return GBP_EINVAL; }
    if (!(p->prior_final_scale > 0.0f) || !std::isfinite(p->prior_final_scale)) { why = "prior_final_scale must be > 0"; return GBP_EINVAL; }
    if (p->prior_anneal_iters < 0) { why = "prior_anneal_iters must be >= 0"; return GBP_EINVAL; }
    if (!(p->anchor_scale >= 0.0f) || !std::isfinite(p->anchor_scale)) { why = "anchor_scale must be >= 0"; return GBP_EINVAL; }
    if (!(p->z_min > 0.0f)) { why = "z_min must be > 0"; return GBP_EINVAL; }
    if (!(p->relin_beta >= 0.0f)) { why = "relin_beta must be >= 0"; return GBP_EINVAL; }
    if (p->relin_interval < 1) { why = "relin_interval must be >= 1"; return GBP_EINVAL; }
    if (p->undamped_iters < 0) { why = "undamped_iters must be >= 0"; return GBP_EINVAL; }
    if (p->check_every < 1) { why = "check_every must be >= 1"; return GBP_EINVAL; }
    if (p->precision_mode < 0 || p->precision_mode > 2) { why = "precision_mode must be 0, 1 or 2"; return GBP_EINVAL; }
    if (p->launch_mode < 0 || p->launch_mode > 2) { why = "launch_mode must be 0, 1 or 2"; return GBP_EINVAL; }
    if (p->damping_mode < 0 || p->damping_mode > 1) { why = "damping_mode must be 0 or 1"; return GBP_EINVAL; }
    if (p->factor_shape < -1 || p->factor_shape >= N_FACTOR_SHAPES) { why = "factor_shape must be -1 .. 5"; return GBP_EINVAL; }
    if (p->fp64_exact_cavity != 0 && p->fp64_exact_cavity != 1) { why = "fp64_exact_cavity must be 0 or 1"; return GBP_EINVAL; }
    if (p->persistent_shape < -1 || p->persistent_shape >= N_PERSISTENT_SHAPES) {
        why = "persistent_shape must be -1 or 0";
        return GBP_EINVAL;
    }
    if (!(p->conv_tol >= 0.0f)) { why = "conv_tol must be >= 0"; return GBP_EINVAL; }
    return GBP_OK;
}

// Sort factors by (landmark, keyframe, caller order); fills the internal
// arrays from the caller's observations.
void order_factors(gbp_graph* g, const std::vector<int32_t>& ok, const std::vector<int32_t>& ol,
                   const std::vector<double>& uv, const std::vector<int32_t>& idx) {
    const int n = (int)ok.size();
    std::vector<int32_t> perm(n);
    std::iota(perm.begin(), perm.end(), 0);
    std::stable_sort(perm.begin(), perm.end(), [&](int a, int b) {
        if (ol[a] != ol[b]) return ol[a] < ol[b];
        return ok[a] < ok[b];
    });
    g->n_f = n;
    g->fk.resize(n);
    g->fm.resize(n);
    g->z.resize(2 * (size_t)n);
    g->obs_index.resize(n);
    for (int i = 0; i < n; ++i) {
        int s = perm[i];
        g->fk[i] = ok[s];
        g->fm[i] = ol[s];
        g->z[2 * i] = uv[2 * s];
        g->z[2 * i + 1] = uv[2 * s + 1];
        g->obs_index[i] = idx[s];
    }
    g->f_of_obs.assign(n, 0);
    for (int i = 0; i < n; ++i) g->f_of_obs[g->obs_index[i]] = i;
}

template <typename R>
void pull_beliefs(gbp_graph* g, std::vector<double>& kb, std::vector<double>& lb, gbp_status& st) {
    DevState<R>& s = state<R>(g);
    std::vector<R> a((size_t)KBEL * g->n_kf), b((size_t)LBEL * g->n_lm);
    cudaError_t e = cudaMemcpyAsync(a.data(), s.kf_bel, sizeof(R) * a.size(), cudaMemcpyDeviceToHost, g->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b.data(), s.lm_bel, sizeof(R) * b.size(), cudaMemcpyDeviceToHost, g->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess) {
        st = cuda_fail(g, e, "belief download");
        return;
    }
    kb.assign(a.begin(), a.end());
    lb.assign(b.begin(), b.end());
    st = GBP_OK;
}

gbp_status download_beliefs(gbp_graph* g, std::vector<double>& kb, std::vector<double>& lb) {
    gbp_status st = GBP_OK;
    if (g->storage) pull_beliefs<double>(g, kb, lb, st);
    else pull_beliefs<float>(g, kb, lb, st);
    return st;
}

// packed lower n x n -> full inverse (double)
bool packed_inverse(int n, const double* P, double* out) {
    double A[36], L[36] = {0};
    for (int i = 0; i < n; ++i)
        for (int j = 0; j <= i; ++j) A[i * n + j] = A[j * n + i] = P[i * (i + 1) / 2 + j];
    for (int j = 0; j < n; ++j) {
        double s = A[j * n + j];
        for (int p = 0; p < j; ++p) s -= L[j * n + p] * L[j * n + p];
        if (!(s > 0.0)) return false;
        L[j * n + j] = std::sqrt(s);
        for (int i = j + 1; i < n; ++i) {
            double t = A[i * n + j];
            for (int p = 0; p < j; ++p) t -= L[i * n + p] * L[j * n + p];
            L[i * n + j] = t / L[j * n + j];
        }
    }
    for (int c = 0; c < n; ++c) {
        double x[6];
        for (int i = 0; i < n; ++i) {
            double s = (i == c) ? 1.0 : 0.0;
            for (int p = 0; p < i; ++p) s -= L[i * n + p] * x[p];
            x[i] = s / L[i * n + i];
        }
        for (int i = n - 1; i >= 0; --i) {
            double s = x[i];
            for (int p = i + 1; p < n; ++p) s -= L[p * n + i] * x[p];
            x[i] = s / L[i * n + i];
        }
        for (int i = 0; i < n; ++i) out[i * n + c] = x[i];
    }
    return true;
}

gbp_status compute_uv_ref(gbp_graph* g, const double* kf_Rt, const double* lm) {
    g->uv_ref.assign(2 * (size_t)g->n_f, 0.0);
    for (int f = 0; f < g->n_f; ++f) {
        const double* Rt = kf_Rt + 12 * (size_t)g->fk[f];
        const double* X = lm + 3 * (size_t)g->fm[f];
        double p[3];
        for (int i = 0; i < 3; ++i) p[i] = Rt[3 * i] * X[0] + Rt[3 * i + 1] * X[1] + Rt[3 * i + 2] * X[2] + Rt[9 + i];
        if (p[2] < g->prm.z_min) {
            g->uv_ref[2 * f] = g->uv_ref[2 * f + 1] = NAN;
        } else {
            g->uv_ref[2 * f] = g->intr.fx * p[0] / p[2] + g->intr.cx;
            g->uv_ref[2 * f + 1] = g->intr.fy * p[1] / p[2] + g->intr.cy;
        }
    }
    return GBP_OK;
}

}  // namespace

// One launch per phase (factor kernel, belief kernel), replayed from a
// captured CUDA graph; with conv_tol > 0 the host checks the largest mean
// change every check_every iterations.
gbp_status iterate_phases(gbp_graph* g, int n, float conv_tol, int* done_out) {
    gbp_status st = ensure_exec(g);
    if (st != GBP_OK) return st;
    const bool check = conv_tol > 0.0f;
    int done = 0;
    if (check && n >= g->prm.check_every) {
        // the whole check blocks in one launch of the device loop; the host
        // loop below takes the rest (fewer than check_every iterations)
        st = ensure_wexec(g);
        if (st != GBP_OK) return st;
        if (g->wexec) {
            const int every = g->prm.check_every, blocks = n / every;
            int32_t tol_bits;
            std::memcpy(&tol_bits, &conv_tol, sizeof tol_bits);
            while_setup_kernel<<<1, 1, 0, g->stream>>>(g->ctl, blocks, tol_bits);
            CK(cudaGetLastError());
            CK(cudaGraphLaunch(g->wexec, g->stream));
            st = read_ctl(g);
            const int runs = blocks - g->h_ctl[CTL_WL_LEFT];
            done = runs * every;
            g->launches += 2 * (int64_t)done + runs + 1;
            *done_out = done;
            if (st != GBP_OK) return st;
            if (last_dmu(g) < conv_tol) return GBP_OK;
        }
    }
    while (done < n) {
        int block = check ? std::min(g->prm.check_every, n - done) : n - done;
        int full = block / GRAPH_CHUNK, rest = block % GRAPH_CHUNK;
        for (int i = 0; i < full; ++i) CK(cudaGraphLaunch(g->exec, g->stream));
        if (rest) {
            cudaError_t e = g->storage ? enqueue_iterations<double>(g, rest, g->stream)
                                       : enqueue_iterations<float>(g, rest, g->stream);
            if (e != cudaSuccess) return cuda_fail(g, e, "kernel launch");
        }
        g->launches += 2 * (int64_t)block;
        done += block;
        *done_out = done;
        if (check) {
            st = read_ctl(g);
            if (st != GBP_OK) return st;
            float dmu;
            dmu = last_dmu(g);
            if (dmu < conv_tol) break;
        }
    }
    return GBP_OK;
}

// One cooperative launch for all n iterations; the convergence test (same
// cadence as above) runs on the device.
gbp_status iterate_persistent(gbp_graph* g, int n, float conv_tol, int* done_out) {
    const int dm = g->prm.damping_mode;
    const int ps = persistent_shape(g);
    const int grid = g->storage ? persistent_grid<double>(g->sd.g, dm, ps) : persistent_grid<float>(g->sf.g, dm, ps);
    if (grid <= 0) return fail(g, GBP_ECUDA, "persistent launch: occupancy query failed");
    cudaError_t e = g->storage
        ? launch_persistent<double>(g->sd.g, make_kparams<double>(g), n, conv_tol, g->prm.check_every, grid, g->stream,
                                    dm, ps)
        : launch_persistent<float>(g->sf.g, make_kparams<float>(g), n, conv_tol, g->prm.check_every, grid, g->stream,
                                   dm, ps);
    if (e != cudaSuccess) return cuda_fail(g, e, "cooperative launch");
    g->launches += 1;
    if (conv_tol > 0.0f) {
        gbp_status st = read_ctl(g);
        *done_out = g->h_ctl[CTL_ITERS_RUN];
        return st;
    }
    *done_out = n;
    return GBP_OK;
}

// Device buffers that make up the iteration state (for snapshots).
template <typename R>
std::vector<std::pair<void*, size_t>> state_buffers(gbp_graph* g) {
    DevState<R>& s = state<R>(g);
    const size_t nf = g->n_f, nk = g->n_kf, nl = g->n_lm;
    return {{s.x0, sizeof(R) * 9 * nf},        {s.tlin, sizeof(int32_t) * nf},   {s.mk, sizeof(R) * KREC * nf},
            {s.mk2, sizeof(R) * KREC * nf},    {s.kj, sizeof(R) * KJ * nf},      {s.lin, sizeof(R) * NLIN * nf},
            {s.ml, sizeof(R) * NML * nf},      {s.kf_bel, sizeof(R) * KBEL * nk}, {s.lm_bel, sizeof(R) * LBEL * nl},
            {s.hist, sizeof(float) * HIST * nf}, {g->ctl, sizeof(int32_t) * CTL_N}};
}

// Slot of every factor's keyframe message: its position in the keyframe's
// CSR list (factors of a keyframe in internal order).
std::vector<int32_t> keyframe_slots(const std::vector<int32_t>& fk, int n_kf) {
    std::vector<int32_t> off(n_kf + 1, 0), kpos(fk.size());
    for (int32_t k : fk) off[k + 1]++;
    for (int v = 0; v < n_kf; ++v) off[v + 1] += off[v];
    for (size_t f = 0; f < fk.size(); ++f) kpos[f] = off[fk[f]]++;
    return kpos;
}

// Incremental SLAM (Sec. 9.2).  The iteration state is carried over factor
// by factor and variable by variable into the rebuilt layout; new variables
// take their prior from their own factors at those factors' linearisation
// points, annealed from this iteration on; new factors are linearised at the
// current means with zero messages.
// The grown factor set's order without a sort: the old factors are in
// (landmark, keyframe, caller) order and every new factor has the new,
// largest keyframe, so each landmark's factors are its old ones followed by
// its new ones in observation order -- what a stable sort of the caller's
// observations by (landmark, keyframe) gives.  src_f receives each factor's
// previous internal index (-1 for a new one).
void order_factors_append(gbp_graph* g, int L1, int K0, int n_obs, const int32_t* obs_lm, const double* obs_uv,
                          std::vector<int32_t>& src_f) {
    const int F0 = g->n_f, F1 = F0 + n_obs;
    std::vector<int32_t> off(L1 + 1, 0), by_lm(n_obs);
    for (int i = 0; i < n_obs; ++i) off[obs_lm[i] + 1]++;
    for (int m = 0; m < L1; ++m) off[m + 1] += off[m];
    {
        std::vector<int32_t> fill(off.begin(), off.end() - 1);
        for (int i = 0; i < n_obs; ++i) by_lm[fill[obs_lm[i]]++] = i;
    }
    std::vector<int32_t> fk(F1), fm(F1), oi(F1);
    std::vector<double> z(2 * (size_t)F1);
    src_f.assign(F1, -1);
    int f = 0, o = 0;
    for (int m = 0; m < L1; ++m) {
        for (; o < F0 && g->fm[o] == m; ++o, ++f) {
            fk[f] = g->fk[o];
            fm[f] = m;
            z[2 * (size_t)f] = g->z[2 * (size_t)o];
            z[2 * (size_t)f + 1] = g->z[2 * (size_t)o + 1];
            oi[f] = g->obs_index[o];
            src_f[f] = o;
        }
        for (int q = off[m]; q < off[m + 1]; ++q, ++f) {
            const int i = by_lm[q];
            fk[f] = K0;
            fm[f] = m;
            z[2 * (size_t)f] = obs_uv[2 * i];
            z[2 * (size_t)f + 1] = obs_uv[2 * i + 1];
            oi[f] = F0 + i;
        }
    }
    g->n_f = F1;
    g->fk.swap(fk);
    g->fm.swap(fm);
    g->z.swap(z);
    g->obs_index.swap(oi);
    g->f_of_obs.assign(F1, 0);
    for (int q = 0; q < F1; ++q) g->f_of_obs[g->obs_index[q]] = q;
}

// Incremental SLAM (Sec. 9.2): the grown graph's layout is built on the host
// from the index arrays alone (no state leaves the device), and the state is
// gathered on the device from the previous layout's buffers
// (relayout_kernel); the host reads back only the control block, the latest
// keyframe's mean and the new variables' prior diagonals.
template <typename R>
gbp_status add_keyframe_impl(gbp_graph* g, const double* kf_Rt_init, int n_new_lm, const double* new_lm_xyz,
                             int n_obs, const int32_t* obs_lm, const double* obs_uv) {
    cudaStream_t st = g->stream;
    const int K0 = g->n_kf, L0 = g->n_lm, F0 = g->n_f;
    const int K1 = K0 + 1, L1 = L0 + n_new_lm, F1 = F0 + n_obs;
    int32_t ctl[CTL_N];
    R mu_last[6];
    {
        DevState<R>& s = state<R>(g);
        CK(cudaMemcpyAsync(ctl, g->ctl, sizeof(int32_t) * CTL_N, cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(mu_last, s.kf_bel + (size_t)KBEL * (K0 - 1) + KB_MU, sizeof(R) * 6, cudaMemcpyDeviceToHost,
                           st));
        CK(cudaStreamSynchronize(st));
    }
    const int t = ctl[CTL_ITER];
    if (ctl[CTL_ERR]) return fail(g, GBP_ESTATE, "graph is in an error state");

    // pose of the new keyframe: given, or the latest keyframe's current estimate
    double Rt[12];
    if (kf_Rt_init) {
        std::copy(kf_Rt_init, kf_Rt_init + 12, Rt);
    } else {
        double w[3] = {double(mu_last[3]), double(mu_last[4]), double(mu_last[5])}, E[9];
        so3_exp_host(w, E);
        const double* Rr = &g->kf_R[9 * (size_t)(K0 - 1)];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) Rt[3 * i + j] = E[3 * i] * Rr[j] + E[3 * i + 1] * Rr[3 + j] + E[3 * i + 2] * Rr[6 + j];
        double c[3];
        for (int i = 0; i < 3; ++i) c[i] = g->kf_c[3 * (K0 - 1) + i] + double(mu_last[i]);
        for (int i = 0; i < 3; ++i) Rt[9 + i] = -(Rt[3 * i] * c[0] + Rt[3 * i + 1] * c[1] + Rt[3 * i + 2] * c[2]);
    }
    double cnew[3];
    for (int i = 0; i < 3; ++i) cnew[i] = -(Rt[i] * Rt[9] + Rt[3 + i] * Rt[10] + Rt[6 + i] * Rt[11]);

    // new variables
    for (int i = 0; i < 9; ++i) g->kf_R.push_back(Rt[i]);
    for (int i = 0; i < 3; ++i) g->kf_c.push_back(cnew[i]);
    g->anchored.push_back(0);
    g->kf_birth.push_back(t);
    for (int j = L0; j < L1; ++j) {
        double X[3];
        if (new_lm_xyz) {
            for (int i = 0; i < 3; ++i) X[i] = new_lm_xyz[3 * (j - L0) + i];
        } else {
            // Sec. 9.2: 1 m depth along the first ray that observes the point
            int o = 0;
            while (obs_lm[o] != j) ++o;
            double pc[3] = {(obs_uv[2 * o] - g->intr.cx) / g->intr.fx, (obs_uv[2 * o + 1] - g->intr.cy) / g->intr.fy, 1.0};
            for (int i = 0; i < 3; ++i) X[i] = cnew[i] + Rt[i] * pc[0] + Rt[3 + i] * pc[1] + Rt[6 + i] * pc[2];
        }
        for (int i = 0; i < 3; ++i) g->lm_ref.push_back(X[i]);
        g->lm_birth.push_back(t);
    }
    g->n_kf = K1;
    g->n_lm = L1;
    std::vector<int32_t> src_f;
    order_factors_append(g, L1, K0, n_obs, obs_lm, obs_uv, src_f);
    g->prob_kf0 = {0, K1};
    g->prob_lm0 = {0, L1};
    g->prob_f0 = {0, F1};
    CK(cudaMemcpy(g->d_prob_f0, g->prob_f0.data(), sizeof(int32_t) * 2, cudaMemcpyHostToDevice));
    g->uv_ref.clear();   // the reference projections no longer cover every factor

    // the previous layout stays alive until its state is gathered, then its
    // buffers go back to the pool for the next addition
    g->headroom = 1.25;
    DevState<R> old = state<R>(g);
    state<R>(g) = DevState<R>();
    int32_t* d_src = nullptr;
    cudaError_t e = dev_alloc(&d_src, (size_t)F1);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_src, src_f.data(), sizeof(int32_t) * (size_t)F1, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) {
        old.release(&g->pool);
        if (d_src) cudaFree(d_src);
        return cuda_fail(g, e, "add_keyframe");
    }
    const RelayoutSrc<R> rs{d_src, F0, L0, t, old.x0, old.tlin, old.ml, old.lin, old.hist, old.kpos, old.kj,
                            (t & 1) ? old.mk2 : old.mk, (t & 1) ? old.mk : old.mk2, old.lm_bel};
    destroy_exec(g);
    gbp_status bst = build_device<R>(g, nullptr, &rs);
    DevState<R>& s = state<R>(g);
    if (bst == GBP_OK) {
        // factor state in the new layout
        e = launch_relayout<R>(s.g, rs, 1, st);
        // priors and beliefs: old variables keep theirs (the prior pass just
        // run covers the new ones), new ones start at their prior at s(0)
        if (e == cudaSuccess) e = cudaMemcpyAsync(s.kf_D, old.kf_D, sizeof(R) * 6 * (size_t)K0, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(s.kf_A, old.kf_A, sizeof(R) * 6 * (size_t)K0, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(s.lm_D, old.lm_D, sizeof(R) * 3 * (size_t)L0, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(s.kf_bel, old.kf_bel, sizeof(R) * KBEL * (size_t)K0, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(s.lm_bel, old.lm_bel, sizeof(R) * LBEL * (size_t)L0, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(s.kjs, 0, sizeof(R) * KJ * (size_t)F1, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(s.mlx, 0, sizeof(R) * 9 * (size_t)F1, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(s.kf_A + 6 * (size_t)K0, 0, sizeof(R) * 6, st);
        std::vector<R> kD(6), lD(3 * (size_t)n_new_lm);
        if (e == cudaSuccess) e = cudaMemcpyAsync(kD.data(), s.kf_D + 6 * (size_t)K0, sizeof(R) * 6, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && n_new_lm)
            e = cudaMemcpyAsync(lD.data(), s.lm_D + 3 * (size_t)L0, sizeof(R) * lD.size(), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e == cudaSuccess) {
            const R s0 = g->prm.prior_anneal_iters > 0 ? R(1) : R(g->prm.prior_final_scale);
            const R isig2 = R(1.0 / (double(g->prm.sigma_px) * double(g->prm.sigma_px)));
            std::vector<R> kbn(KBEL), lbn(LBEL * (size_t)n_new_lm, R(0));
            R pd[6];
            for (int i = 0; i < 6; ++i) pd[i] = s0 * kD[i] * isig2;
            kf_prior_record_host<R>(pd, kbn.data());
            for (int j = 0; j < n_new_lm; ++j)
                for (int i = 0; i < 3; ++i) lbn[(size_t)LBEL * j + i * (i + 1) / 2 + i] = s0 * lD[3 * (size_t)j + i] * isig2;
            e = cudaMemcpyAsync(s.kf_bel + (size_t)KBEL * K0, kbn.data(), sizeof(R) * KBEL, cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess && n_new_lm)
                e = cudaMemcpyAsync(s.lm_bel + (size_t)LBEL * L0, lbn.data(), sizeof(R) * lbn.size(),
                                    cudaMemcpyHostToDevice, st);
            // the control block as it was (the prior pass leaves it alone; kept
            // explicit so that the iteration count and flags carry over)
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(g->ctl, ctl, sizeof(int32_t) * CTL_N, cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        }
    }
    old.release(&g->pool);
    cudaFree(d_src);
    if (bst != GBP_OK) return bst;
    if (e != cudaSuccess) return cuda_fail(g, e, "add_keyframe");
    return GBP_OK;
}

// Record schedule: n iterations with the fixed damping schedule, one launch
// per phase, each writing its n_f feature rows and damping targets.
template <typename R>
gbp_status record_iterations(gbp_graph* g, int n, float* X, float* T) {
    DevState<R>& s = state<R>(g);
    DevGraph<R> d = s.g;
    d.eta_inf = s.eta_inf;
    const KParams<R> kp = make_kparams<R>(g);
    for (int i = 0; i < n; ++i) {
        d.rec_X = X + (size_t)i * g->n_f * N_FEAT;
        d.rec_T = T + (size_t)i * g->n_f;
        CK(launch_factor<R>(d, kp, g->stream, DAMP_RECORD, g->pdl));
        CK(launch_belief<R>(d, kp, g->stream, g->pdl));
    }
    g->launches += 2 * (int64_t)n;
    return GBP_OK;
}

// ==========================================================================
// C ABI

extern "C" {

void gbp_default_params(gbp_params* p) {
    if (!p) return;
    p->damping = 0.4f;
    p->huber_nsigma = 0.0f;
    p->sigma_px = 1.0f;
    p->iterations = 200;
    p->conv_tol = 0.0f;
    p->check_every = 16;
    p->prior_final_scale = 0.01f;
    p->prior_anneal_iters = 10;
    p->anchor_scale = 1000.0f;
    p->z_min = 0.05f;
    p->relin_beta = 0.01f;
    p->relin_interval = 10;
    p->undamped_iters = 8;
    p->fp64_pivot_ratio = 1e-6f;
    p->precision_mode = 0;
    p->linear = 0;
    p->launch_mode = 0;
    p->damping_mode = 0;
    p->factor_shape = -1;
    p->persistent_shape = -1;
    p->fp64_exact_cavity = 0;
}

const char* gbp_status_string(gbp_status s) {
    switch (s) {
        case GBP_OK: return "ok";
        case GBP_EINVAL: return "invalid argument";
        case GBP_ENOMEM: return "out of memory";
        case GBP_ECUDA: return "CUDA error";
        case GBP_EDIVERGED: return "diverged";
        case GBP_ETIMEOUT: return "timeout";
        case GBP_ESTATE: return "invalid state";
    }
    return "unknown status";
}

const char* gbp_last_error(const gbp_graph* g) { return g ? g->err.c_str() : "null graph"; }

namespace {

// Shared body of gbp_create_graph and gbp_create_batch.  prob_kf0 / prob_lm0
// hold the first keyframe / landmark of every problem plus the totals.
gbp_status create_impl(const gbp_intrinsics* intr, int32_t n_kf, const double* kf_Rt, int32_t n_lm,
                       const double* lm_xyz, int32_t n_obs, const int32_t* obs_kf, const int32_t* obs_lm,
                       const double* obs_uv, int32_t n_anchor, const int32_t* anchor_kf,
                       const std::vector<int32_t>& prob_kf0, const std::vector<int32_t>& prob_lm0, void* cuda_stream,
                       gbp_graph** out) {
    if (!out) return GBP_EINVAL;
    *out = nullptr;
    if (!intr || n_kf < 0 || n_lm < 0 || n_obs < 0 || n_anchor < 0) return GBP_EINVAL;
    if ((n_kf && !kf_Rt) || (n_lm && !lm_xyz) || (n_obs && (!obs_kf || !obs_lm || !obs_uv)) ||
        (n_anchor && !anchor_kf))
        return GBP_EINVAL;
    if (!std::isfinite(intr->fx) || !std::isfinite(intr->fy) || !std::isfinite(intr->cx) ||
        !std::isfinite(intr->cy) || intr->fx == 0.0 || intr->fy == 0.0)
        return GBP_EINVAL;
    if (!finite_all(kf_Rt, 12 * (size_t)n_kf) || !finite_all(lm_xyz, 3 * (size_t)n_lm) ||
        !finite_all(obs_uv, 2 * (size_t)n_obs))
        return GBP_EINVAL;
    for (int i = 0; i < n_obs; ++i)
        if (obs_kf[i] < 0 || obs_kf[i] >= n_kf || obs_lm[i] < 0 || obs_lm[i] >= n_lm) return GBP_EINVAL;
    for (int i = 0; i < n_anchor; ++i)
        if (anchor_kf[i] < 0 || anchor_kf[i] >= n_kf) return GBP_EINVAL;

    gbp_graph* g = new (std::nothrow) gbp_graph();
    if (!g) return GBP_ENOMEM;
    (void)cudaGetLastError();   // an error left by an unrelated earlier call is not ours to report
    g->intr = *intr;
    gbp_default_params(&g->prm);
    g->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    g->n_kf = n_kf;
    g->n_lm = n_lm;
    g->prob_kf0 = prob_kf0;
    g->prob_lm0 = prob_lm0;
    g->kf_R.resize(9 * (size_t)n_kf);
    g->kf_c.resize(3 * (size_t)n_kf);
    for (int v = 0; v < n_kf; ++v) {
        const double* Rt = kf_Rt + 12 * (size_t)v;
        for (int i = 0; i < 9; ++i) g->kf_R[9 * v + i] = Rt[i];
        // camera centre c = -R^T t
        for (int i = 0; i < 3; ++i) g->kf_c[3 * v + i] = -(Rt[i] * Rt[9] + Rt[3 + i] * Rt[10] + Rt[6 + i] * Rt[11]);
    }
    g->lm_ref.assign(lm_xyz, lm_xyz + 3 * (size_t)n_lm);
    g->kf_birth.assign(n_kf, 0);
    g->lm_birth.assign(n_lm, 0);
    g->anchored.assign(n_kf, 0);
    for (int i = 0; i < n_anchor; ++i) g->anchored[anchor_kf[i]] = 1;
    // every observed point must be in front of its camera at the initial values
    for (int i = 0; i < n_obs; ++i) {
        const double* Rt = kf_Rt + 12 * (size_t)obs_kf[i];
        const double* X = lm_xyz + 3 * (size_t)obs_lm[i];
        double pz = Rt[6] * X[0] + Rt[7] * X[1] + Rt[8] * X[2] + Rt[11];
        if (!(pz >= g->prm.z_min)) {
            char buf[128];
            snprintf(buf, sizeof buf, "observation %d: point depth %.4g below z_min at the initial values", i, pz);
            g->err = buf;
            delete g;
            return GBP_EINVAL;
        }
    }
    {
        std::vector<int32_t> ok(obs_kf, obs_kf + n_obs), ol(obs_lm, obs_lm + n_obs), idx(n_obs);
        std::vector<double> uv(obs_uv, obs_uv + 2 * (size_t)n_obs);
        std::iota(idx.begin(), idx.end(), 0);
        order_factors(g, ok, ol, uv, idx);
        // factors are sorted by landmark, and each problem's landmarks are
        // contiguous: a problem's factors are one contiguous range
        const int np = (int)g->prob_lm0.size() - 1;
        g->prob_f0.assign(np + 1, 0);
        for (int p = 0; p <= np; ++p)
            g->prob_f0[p] = (int32_t)(std::lower_bound(g->fm.begin(), g->fm.end(), g->prob_lm0[p]) - g->fm.begin());
    }
    cudaError_t e = cudaStreamCreateWithFlags(&g->capture, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&g->ctl), sizeof(int32_t) * CTL_N);
    g->n_partials = metrics_blocks(g->n_f);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&g->partials), sizeof(double) * 6 * g->n_partials);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&g->met), sizeof(double) * MET_N);
    if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void**>(&g->h_ctl), sizeof(int32_t) * CTL_N);
    if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void**>(&g->h_met), sizeof(double) * MET_N);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&g->d_prob_f0), sizeof(int32_t) * g->prob_f0.size());
    if (e == cudaSuccess)
        e = cudaMemcpy(g->d_prob_f0, g->prob_f0.data(), sizeof(int32_t) * g->prob_f0.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        gbp_destroy_graph(g);
        return e == cudaErrorMemoryAllocation ? GBP_ENOMEM : GBP_ECUDA;
    }
    gbp_status st = ensure_built(g);
    if (st != GBP_OK) {
        gbp_destroy_graph(g);
        return st;
    }
    *out = g;
    return GBP_OK;
}

}  // namespace

gbp_status gbp_create_graph(const gbp_intrinsics* intr, int32_t n_kf, const double* kf_Rt, int32_t n_lm,
                            const double* lm_xyz, int32_t n_obs, const int32_t* obs_kf, const int32_t* obs_lm,
                            const double* obs_uv, int32_t n_anchor, const int32_t* anchor_kf, void* cuda_stream,
                            gbp_graph** out) {
    if (n_kf < 0 || n_lm < 0) return GBP_EINVAL;
    return create_impl(intr, n_kf, kf_Rt, n_lm, lm_xyz, n_obs, obs_kf, obs_lm, obs_uv, n_anchor, anchor_kf,
                       {0, n_kf}, {0, n_lm}, cuda_stream, out);
}

gbp_status gbp_create_batch(const gbp_intrinsics* intr, int32_t n_problems, const gbp_problem_desc* probs,
                            void* cuda_stream, gbp_graph** out) {
    if (!out) return GBP_EINVAL;
    *out = nullptr;
    if (!intr || n_problems < 0 || (n_problems && !probs)) return GBP_EINVAL;
    std::vector<int32_t> kf0(1, 0), lm0(1, 0);
    int64_t nk = 0, nl = 0, no = 0, na = 0;
    for (int p = 0; p < n_problems; ++p) {
        const gbp_problem_desc& d = probs[p];
        if (d.n_kf < 0 || d.n_lm < 0 || d.n_obs < 0 || d.n_anchor < 0) return GBP_EINVAL;
        if ((d.n_kf && !d.kf_Rt) || (d.n_lm && !d.lm_xyz) || (d.n_obs && (!d.obs_kf || !d.obs_lm || !d.obs_uv)) ||
            (d.n_anchor && !d.anchor_kf))
            return GBP_EINVAL;
        for (int i = 0; i < d.n_obs; ++i)
            if (d.obs_kf[i] < 0 || d.obs_kf[i] >= d.n_kf || d.obs_lm[i] < 0 || d.obs_lm[i] >= d.n_lm) return GBP_EINVAL;
        for (int i = 0; i < d.n_anchor; ++i)
            if (d.anchor_kf[i] < 0 || d.anchor_kf[i] >= d.n_kf) return GBP_EINVAL;
        nk += d.n_kf;
        nl += d.n_lm;
        no += d.n_obs;
        na += d.n_anchor;
        if (nk > INT32_MAX || nl > INT32_MAX || no > INT32_MAX) return GBP_EINVAL;
        kf0.push_back((int32_t)nk);
        lm0.push_back((int32_t)nl);
    }
    std::vector<double> kf(12 * (size_t)nk), lm(3 * (size_t)nl), uv(2 * (size_t)no);
    std::vector<int32_t> ok(no), ol(no), an(na);
    size_t o = 0, a = 0;
    for (int p = 0; p < n_problems; ++p) {
        const gbp_problem_desc& d = probs[p];
        std::copy(d.kf_Rt, d.kf_Rt + 12 * (size_t)d.n_kf, kf.begin() + 12 * (size_t)kf0[p]);
        std::copy(d.lm_xyz, d.lm_xyz + 3 * (size_t)d.n_lm, lm.begin() + 3 * (size_t)lm0[p]);
        for (int i = 0; i < d.n_obs; ++i, ++o) {
            ok[o] = d.obs_kf[i] + kf0[p];
            ol[o] = d.obs_lm[i] + lm0[p];
            uv[2 * o] = d.obs_uv[2 * i];
            uv[2 * o + 1] = d.obs_uv[2 * i + 1];
        }
        for (int i = 0; i < d.n_anchor; ++i, ++a) an[a] = d.anchor_kf[i] + kf0[p];
    }
    return create_impl(intr, (int32_t)nk, kf.data(), (int32_t)nl, lm.data(), (int32_t)no, ok.data(), ol.data(),
                       uv.data(), (int32_t)na, an.data(), kf0, lm0, cuda_stream, out);
}

gbp_status gbp_get_batch_info(const gbp_graph* g, int32_t* n_problems, int32_t* kf_offsets, int32_t* lm_offsets,
                              int32_t* obs_counts) {
    if (!g) return GBP_EINVAL;
    const int np = (int)g->prob_kf0.size() - 1;
    if (n_problems) *n_problems = np;
    for (int p = 0; p <= np; ++p) {
        if (kf_offsets) kf_offsets[p] = g->prob_kf0[p];
        if (lm_offsets) lm_offsets[p] = g->prob_lm0[p];
        if (obs_counts && p < np) obs_counts[p] = g->prob_f0[p + 1] - g->prob_f0[p];
    }
    return GBP_OK;
}

gbp_status gbp_get_problem_are(const gbp_graph* cg, double* are, int32_t* n_are, int32_t* huber) {
    gbp_graph* g = const_cast<gbp_graph*>(cg);
    if (!g || !are) return GBP_EINVAL;
    const int np = (int)g->prob_kf0.size() - 1;
    if (np == 0) return GBP_OK;
    double* d_out = nullptr;
    CK(cudaMalloc(reinterpret_cast<void**>(&d_out), sizeof(double) * 3 * np));
    cudaError_t e = g->storage
        ? launch_problem_metrics<double>(g->sd.g, make_kparams<double>(g), g->d_prob_f0, np, d_out, g->stream)
        : launch_problem_metrics<float>(g->sf.g, make_kparams<float>(g), g->d_prob_f0, np, d_out, g->stream);
    std::vector<double> h(3 * (size_t)np);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), d_out, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, g->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    cudaFree(d_out);
    if (e != cudaSuccess) return cuda_fail(g, e, "problem metrics");
    for (int p = 0; p < np; ++p) {
        are[p] = h[3 * p + 1] > 0 ? h[3 * p] / h[3 * p + 1] : 0.0;
        if (n_are) n_are[p] = (int32_t)h[3 * p + 1];
        if (huber) huber[p] = (int32_t)h[3 * p + 2];
    }
    return read_ctl(g);
}

gbp_status gbp_set_params(gbp_graph* g, const gbp_params* p) {
    if (!g || !p) return GBP_EINVAL;
    std::string why;
    if (check_params(p, why) != GBP_OK) return fail(g, GBP_EINVAL, why);
    bool sigma_changed = p->sigma_px != g->prm.sigma_px;
    if (p->precision_mode != g->prm.precision_mode || p->damping_mode != g->prm.damping_mode) {
        g->tuned_mode = 0;
        g->tuned_fshape = g->tuned_pshape = -1;
    }
    g->prm = *p;
    destroy_exec(g);
    (void)sigma_changed;   // priors are stored at sigma = 1 and scaled in the kernels
    gbp_status st = ensure_built(g);
    if (st != GBP_OK) return st;
    return g->storage ? upload_prior_table<double>(g) : upload_prior_table<float>(g);
}

gbp_status gbp_get_params(const gbp_graph* g, gbp_params* out) {
    if (!g || !out) return GBP_EINVAL;
    *out = g->prm;
    return GBP_OK;
}

gbp_status gbp_reset(gbp_graph* g) {
    if (!g) return GBP_EINVAL;
    gbp_status st = ensure_built(g);
    if (st != GBP_OK) return st;
    // back to iteration 0: every variable counts as present from the start
    if (std::any_of(g->kf_birth.begin(), g->kf_birth.end(), [](int32_t b) { return b != 0; }) ||
        std::any_of(g->lm_birth.begin(), g->lm_birth.end(), [](int32_t b) { return b != 0; })) {
        std::fill(g->kf_birth.begin(), g->kf_birth.end(), 0);
        std::fill(g->lm_birth.begin(), g->lm_birth.end(), 0);
        int32_t* kb = g->storage ? g->sd.kf_birth : g->sf.kf_birth;
        int32_t* lb = g->storage ? g->sd.lm_birth : g->sf.lm_birth;
        if (g->n_kf) CK(cudaMemcpy(kb, g->kf_birth.data(), sizeof(int32_t) * g->n_kf, cudaMemcpyHostToDevice));
        if (g->n_lm) CK(cudaMemcpy(lb, g->lm_birth.data(), sizeof(int32_t) * g->n_lm, cudaMemcpyHostToDevice));
    }
    return g->storage ? reset_state<double>(g) : reset_state<float>(g);
}

// The auto launch mode's choices, per device and graph shape.  Every
// candidate gives bitwise identical results, so a graph whose device,
// storage, precision mode, damping schedule and sizes (keyframes, points, factors, warp
// tiles, problems) match a graph already tuned in this process takes that
// choice instead of timing the candidates again (gbp_autotune, called
// explicitly, always times them and records its choice here).
namespace {
using TuneKey = std::tuple<int, int, int, int, int, int, int, int, int>;
struct TuneVal {
    int mode, fshape, pshape;
    gbp_tuning tuning;
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneVal> g_tune_cache;
constexpr size_t TUNE_CACHE_MAX = 256;   // graph shapes remembered at once

bool tune_key(const gbp_graph* g, TuneKey& key) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    const int n_tiles = g->storage ? g->sd.g.n_tiles : g->sf.g.n_tiles;
    key = TuneKey(dev, g->storage, g->prm.precision_mode, g->prm.damping_mode, g->n_kf, g->n_lm, g->n_f, n_tiles,
                  (int)g->prob_f0.size());
    return true;
}

bool tune_cache_lookup(gbp_graph* g) {
    TuneKey key;
    if (!tune_key(g, key)) return false;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it == g_tune_cache.end()) return false;
    g->tuned_mode = it->second.mode;
    g->tuned_fshape = it->second.fshape;
    g->tuned_pshape = it->second.pshape;
    g->tuning = it->second.tuning;
    destroy_exec(g);   // a graph recorded before with the default shapes
    return true;
}

void tune_cache_store(const gbp_graph* g) {
    TuneKey key;
    if (!tune_key(g, key)) return;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    if (g_tune_cache.size() >= TUNE_CACHE_MAX && !g_tune_cache.count(key)) g_tune_cache.clear();   // bounded
    g_tune_cache[key] = TuneVal{g->tuned_mode, g->tuned_fshape, g->tuned_pshape, g->tuning};
}
}  // namespace

gbp_status gbp_iterate(gbp_graph* g, int32_t n_iters, int32_t* iters_done) {
    if (iters_done) *iters_done = 0;
    if (!g) return GBP_EINVAL;
    gbp_status st = ensure_built(g);
    if (st != GBP_OK) return st;
    int n = n_iters > 0 ? n_iters : g->prm.iterations;
    if (g->part_lm1 >= 0) return fail(g, GBP_ESTATE, "a partitioned graph iterates with gbp_split_phase");
    if (g->n_f == 0 && g->n_kf == 0 && g->n_lm == 0) return GBP_OK;
    if (g->prm.damping_mode == 1 && !g->has_model)
        return fail(g, GBP_ESTATE, "damping_mode 1 needs a network (gbp_set_damping_model)");
    int mode = g->prm.launch_mode;
    if (mode == 0) {
        if (!g->tuned_mode && !tune_cache_lookup(g)) {
            st = gbp_autotune(g, 8, nullptr, nullptr);
            if (st != GBP_OK) return st;
        }
        mode = g->tuned_mode;
    }
    int done = 0;
    g->last_mode = mode;
    st = mode == 1 ? iterate_persistent(g, n, g->prm.conv_tol, &done) : iterate_phases(g, n, g->prm.conv_tol, &done);
    if (iters_done) *iters_done = done;
    return st;
}

gbp_status gbp_get_means(const gbp_graph* cg, double* kf_mu, double* lm_mu) {
    gbp_graph* g = const_cast<gbp_graph*>(cg);
    if (!g || (g->n_kf && !kf_mu) || (g->n_lm && !lm_mu)) return GBP_EINVAL;
    std::vector<double> kb, lb;
    gbp_status st = download_beliefs(g, kb, lb);
    if (st != GBP_OK) return st;
    for (int v = 0; v < g->n_kf; ++v)
        for (int i = 0; i < 6; ++i) kf_mu[6 * v + i] = kb[(size_t)KBEL * v + KB_MU + i];
    for (int v = 0; v < g->n_lm; ++v)
        for (int i = 0; i < 3; ++i) lm_mu[3 * v + i] = lb[(size_t)LBEL * v + 9 + i];
    return read_ctl(g);
}

gbp_status gbp_get_beliefs(const gbp_graph* cg, double* kf_Rt, double* lm_xyz, double* kf_cov, double* lm_cov) {
    gbp_graph* g = const_cast<gbp_graph*>(cg);
    if (!g || (g->n_kf && !kf_Rt) || (g->n_lm && !lm_xyz)) return GBP_EINVAL;
    std::vector<double> kb, lb;
    gbp_status st = download_beliefs(g, kb, lb);
    if (st != GBP_OK) return st;
    for (int v = 0; v < g->n_kf; ++v) {
        const double* mu = &kb[(size_t)KBEL * v + KB_MU];
        double E[9], R[9], c[3];
        so3_exp_host(mu + 3, E);
        const double* Rr = &g->kf_R[9 * (size_t)v];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                R[3 * i + j] = E[3 * i] * Rr[j] + E[3 * i + 1] * Rr[3 + j] + E[3 * i + 2] * Rr[6 + j];
        for (int i = 0; i < 3; ++i) c[i] = g->kf_c[3 * v + i] + mu[i];
        double* o = kf_Rt + 12 * (size_t)v;
        for (int i = 0; i < 9; ++i) o[i] = R[i];
        for (int i = 0; i < 3; ++i) o[9 + i] = -(R[3 * i] * c[0] + R[3 * i + 1] * c[1] + R[3 * i + 2] * c[2]);
        if (kf_cov && !packed_inverse(6, &kb[(size_t)KBEL * v + KB_LAM], kf_cov + 36 * (size_t)v))
            return fail(g, GBP_EDIVERGED, "keyframe belief not positive definite");
    }
    for (int v = 0; v < g->n_lm; ++v) {
        for (int i = 0; i < 3; ++i) lm_xyz[3 * v + i] = g->lm_ref[3 * v + i] + lb[(size_t)LBEL * v + 9 + i];
        if (lm_cov && !packed_inverse(3, &lb[(size_t)LBEL * v], lm_cov + 9 * (size_t)v))
            return fail(g, GBP_EDIVERGED, "landmark belief not positive definite");
    }
    return read_ctl(g);
}

gbp_status gbp_set_reference(gbp_graph* g, const double* ref_kf_Rt, const double* ref_lm) {
    if (!g) return GBP_EINVAL;
    if (!ref_kf_Rt || !ref_lm) {
        g->uv_ref.clear();
    } else {
        if (!finite_all(ref_kf_Rt, 12 * (size_t)g->n_kf) || !finite_all(ref_lm, 3 * (size_t)g->n_lm))
            return fail(g, GBP_EINVAL, "reference solution not finite");
        compute_uv_ref(g, ref_kf_Rt, ref_lm);
    }
    // upload into the current storage
    destroy_exec(g);
    if (g->storage) {
        DevState<double>& s = g->sd;
        if (s.uv_ref) cudaFree(s.uv_ref);
        s.uv_ref = nullptr;
        s.g.uv_ref = nullptr;
        if (!g->uv_ref.empty()) {
            CK(dev_alloc(&s.uv_ref, g->uv_ref.size()));
            CK(cudaMemcpyAsync(s.uv_ref, g->uv_ref.data(), sizeof(double) * g->uv_ref.size(), cudaMemcpyHostToDevice, g->stream));
            s.g.uv_ref = s.uv_ref;
        }
    } else {
        DevState<float>& s = g->sf;
        if (s.uv_ref) cudaFree(s.uv_ref);
        s.uv_ref = nullptr;
        s.g.uv_ref = nullptr;
        if (!g->uv_ref.empty()) {
            std::vector<float> u(g->uv_ref.begin(), g->uv_ref.end());
            CK(dev_alloc(&s.uv_ref, u.size()));
            CK(cudaMemcpyAsync(s.uv_ref, u.data(), sizeof(float) * u.size(), cudaMemcpyHostToDevice, g->stream));
            s.g.uv_ref = s.uv_ref;
        }
    }
    CK(cudaStreamSynchronize(g->stream));
    return GBP_OK;
}

gbp_status gbp_get_stats(const gbp_graph* cg, gbp_stats* out) {
    gbp_graph* g = const_cast<gbp_graph*>(cg);
    if (!g || !out) return GBP_EINVAL;
    std::memset(out, 0, sizeof *out);
    cudaError_t e = g->storage
        ? launch_metrics<double>(g->sd.g, make_kparams<double>(g), g->partials, g->n_partials, g->met, g->stream)
        : launch_metrics<float>(g->sf.g, make_kparams<float>(g), g->partials, g->n_partials, g->met, g->stream);
    if (e != cudaSuccess) return cuda_fail(g, e, "metrics");
    CK(cudaMemcpyAsync(g->h_met, g->met, sizeof(double) * MET_N, cudaMemcpyDeviceToHost, g->stream));
    gbp_status st = read_ctl(g);   // synchronises
    out->iterations = g->h_ctl[CTL_ITER];
    out->max_dmu = last_dmu(g);
    out->are = g->h_met[MET_ARE];
    out->are_ref = g->h_met[MET_ARE_REF];
    out->n_are = (int32_t)g->h_met[MET_N_ARE];
    out->huber_count = (int32_t)g->h_met[MET_HUBER];
    out->fp64_fallbacks = g->h_ctl[CTL_FALLBACKS];
    out->relinearisations = g->h_ctl[CTL_RELINS];
    out->held_messages = g->h_ctl[CTL_HELD];
    out->fp64_resums = g->h_ctl[CTL_RESUMS];
    out->launch_mode = g->last_mode;
    out->kernel_launches = g->launches;
    return st;
}

gbp_status gbp_get_relin_iters(const gbp_graph* cg, int32_t* tlin) {
    gbp_graph* g = const_cast<gbp_graph*>(cg);
    if (!g || (g->n_f && !tlin)) return GBP_EINVAL;
    std::vector<int32_t> t(g->n_f);
    if (g->n_f) {
        const int32_t* d = g->storage ? g->sd.tlin : g->sf.tlin;
        CK(cudaMemcpyAsync(t.data(), d, sizeof(int32_t) * t.size(), cudaMemcpyDeviceToHost, g->stream));
        CK(cudaStreamSynchronize(g->stream));
    }
    for (int f = 0; f < g->n_f; ++f) tlin[g->obs_index[f]] = t[f];
    return read_ctl(g);
}

gbp_status gbp_get_residuals(const gbp_graph* cg, double* err) {
    gbp_graph* g = const_cast<gbp_graph*>(cg);
    if (!g || (g->n_f && !err)) return GBP_EINVAL;
    if (g->n_f == 0) return GBP_OK;
    double* d = nullptr;
    CK(cudaMalloc(reinterpret_cast<void**>(&d), sizeof(double) * g->n_f));
    cudaError_t e = g->storage ? launch_residuals<double>(g->sd.g, make_kparams<double>(g), d, g->stream)
                               : launch_residuals<float>(g->sf.g, make_kparams<float>(g), d, g->stream);
    std::vector<double> h(g->n_f);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), d, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, g->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    cudaFree(d);
    if (e != cudaSuccess) return cuda_fail(g, e, "residuals");
    for (int f = 0; f < g->n_f; ++f) err[g->obs_index[f]] = h[f];
    return read_ctl(g);
}

gbp_status gbp_get_sizes(const gbp_graph* g, int32_t* n_kf, int32_t* n_lm, int32_t* n_obs) {
    if (!g) return GBP_EINVAL;
    if (n_kf) *n_kf = g->n_kf;
    if (n_lm) *n_lm = g->n_lm;
    if (n_obs) *n_obs = g->n_f;
    return GBP_OK;
}

gbp_status gbp_profile_iterations(gbp_graph* g, int32_t n_iters, double* ms_out) {
    if (!g || !ms_out || n_iters <= 0) return GBP_EINVAL;
    gbp_status st = ensure_built(g);
    if (st != GBP_OK) return st;
    if (g->prm.damping_mode == 1 && !g->has_model)
        return fail(g, GBP_ESTATE, "damping_mode 1 needs a network (gbp_set_damping_model)");
    int mode = g->prm.launch_mode ? g->prm.launch_mode : (g->tuned_mode ? g->tuned_mode : 2);
    cudaEvent_t ev[2] = {nullptr, nullptr};
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaEventCreate(&ev[i]);
    if (e != cudaSuccess) return cuda_fail(g, e, "cudaEventCreate");
    // (a) whole iterations in the current launch mode, from reset
    st = g->storage ? reset_state<double>(g) : reset_state<float>(g);
    int done = 0;
    if (st == GBP_OK && mode == 2) st = ensure_exec(g);
    if (st == GBP_OK) {
        cudaEventRecord(ev[0], g->stream);
        st = mode == 1 ? iterate_persistent(g, n_iters, 0.0f, &done) : iterate_phases(g, n_iters, 0.0f, &done);
        cudaEventRecord(ev[1], g->stream);
    }
    float ms_iter = 0.f;
    if (st == GBP_OK) {
        e = cudaStreamSynchronize(g->stream);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms_iter, ev[0], ev[1]);
    }
    // (b) the factor kernel alone, replayed with its outputs in scratch
    const size_t rs = g->storage ? sizeof(double) : sizeof(float);
    void* scratch[3] = {nullptr, nullptr, nullptr};
    const size_t sizes[3] = {rs * KREC * std::max(g->n_f, 1), rs * NML * std::max(g->n_f, 1),
                             rs * LBEL * std::max(g->n_lm, 1)};
    cudaGraphExec_t ex = nullptr;
    float ms_fac = 0.f;
    if (st == GBP_OK && e == cudaSuccess) {
        for (int i = 0; i < 3 && e == cudaSuccess; ++i) e = cudaMalloc(&scratch[i], sizes[i]);
        DevGraph<float> pf = g->sf.g;
        DevGraph<double> pd = g->sd.g;
        pf.mk_redirect = static_cast<float*>(scratch[0]);
        pf.ml_out = static_cast<float*>(scratch[1]);
        pf.lm_bel_out = static_cast<float*>(scratch[2]);
        pd.mk_redirect = static_cast<double*>(scratch[0]);
        pd.ml_out = static_cast<double*>(scratch[1]);
        pd.lm_bel_out = static_cast<double*>(scratch[2]);
        const KParams<float> kf_ = make_kparams<float>(g);
        const KParams<double> kd_ = make_kparams<double>(g);
        cudaGraph_t graph = nullptr;
        if (e == cudaSuccess) e = cudaStreamBeginCapture(g->capture, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t le = cudaSuccess;
            for (int i = 0; i < n_iters && le == cudaSuccess; ++i)
                le = g->storage ? launch_factor<double>(pd, kd_, g->capture, g->prm.damping_mode, false, 0)
                                : launch_factor<float>(pf, kf_, g->capture, g->prm.damping_mode, false,
                                                       factor_shape(g));
            e = cudaStreamEndCapture(g->capture, &graph);
            if (le != cudaSuccess) e = le;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&ex, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e == cudaSuccess) {
            cudaGraphLaunch(ex, g->stream);
            cudaEventRecord(ev[0], g->stream);
            cudaGraphLaunch(ex, g->stream);
            cudaEventRecord(ev[1], g->stream);
            e = cudaStreamSynchronize(g->stream);
        }
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms_fac, ev[0], ev[1]);
    }
    for (auto& x : ev)
        if (x) cudaEventDestroy(x);
    if (ex) cudaGraphExecDestroy(ex);
    for (auto& p : scratch)
        if (p) cudaFree(p);
    if (st != GBP_OK) return st;
    if (e != cudaSuccess) return cuda_fail(g, e, "profile");
    ms_out[0] = double(ms_iter) / n_iters;
    ms_out[1] = double(ms_fac) / n_iters;
    st = read_ctl(g);
    if (st != GBP_OK) return st;
    return g->storage ? reset_state<double>(g) : reset_state<float>(g);
}

gbp_status gbp_autotune(gbp_graph* g, int32_t n_trial, int32_t* chosen, double* ms_out) {
    if (!g || n_trial <= 0) return GBP_EINVAL;
    gbp_status st = ensure_built(g);
    if (st != GBP_OK) return st;
    if (g->prm.damping_mode == 1 && !g->has_model)
        return fail(g, GBP_ESTATE, "damping_mode 1 needs a network (gbp_set_damping_model)");
    // candidates: (mode, shape); only the FP32 fixed schedule has several shapes
    std::vector<std::pair<int, int>> cand;
    const int np = tunable(g) ? n_persistent_shapes(g) : 1, nf = tunable(g) ? N_FACTOR_SHAPES : 1;
    for (int s = 0; s < np; ++s) cand.push_back({1, s});
    for (int s = 0; s < nf; ++s) cand.push_back({2, s});
    auto bufs = g->storage ? state_buffers<double>(g) : state_buffers<float>(g);
    std::vector<void*> snap(bufs.size(), nullptr);
    cudaError_t e = cudaSuccess;
    for (size_t i = 0; i < bufs.size() && e == cudaSuccess; ++i) {
        e = cudaMalloc(&snap[i], std::max<size_t>(bufs[i].second, 1));
        if (e == cudaSuccess) e = cudaMemcpyAsync(snap[i], bufs[i].first, bufs[i].second, cudaMemcpyDeviceToDevice, g->stream);
    }
    cudaEvent_t ev[2] = {nullptr, nullptr};
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaEventCreate(&ev[i]);
    const gbp_params saved = g->prm;
    std::vector<double> ms(cand.size(), -1.0);
    for (size_t c = 0; c < cand.size() && e == cudaSuccess; ++c) {
        const int mode = cand[c].first;
        g->prm.launch_mode = mode;
        g->prm.factor_shape = mode == 2 ? cand[c].second : 0;
        g->prm.persistent_shape = mode == 1 ? cand[c].second : 0;
        destroy_exec(g);
        if (mode == 2) {
            st = ensure_exec(g);
            if (st != GBP_OK) break;
        }
        int done = 0;
        // one untimed warm run, then the timed run, each from the snapshot
        for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
            cudaEventRecord(ev[0], g->stream);
            gbp_status ms_st = mode == 1 ? iterate_persistent(g, n_trial, 0.0f, &done)
                                         : iterate_phases(g, n_trial, 0.0f, &done);
            cudaEventRecord(ev[1], g->stream);
            e = cudaStreamSynchronize(g->stream);
            if (ms_st != GBP_OK) {
                g->err.clear();
                cudaGetLastError();
                e = cudaSuccess;
                ms[c] = -1.0;
            } else if (e == cudaSuccess && rep == 1) {
                float t = 0.f;
                e = cudaEventElapsedTime(&t, ev[0], ev[1]);
                ms[c] = double(t) / n_trial;
            }
            for (size_t i = 0; i < bufs.size() && e == cudaSuccess; ++i)
                e = cudaMemcpyAsync(bufs[i].first, snap[i], bufs[i].second, cudaMemcpyDeviceToDevice, g->stream);
            if (ms_st != GBP_OK) break;
        }
    }
    g->prm = saved;
    destroy_exec(g);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    for (auto& x : ev)
        if (x) cudaEventDestroy(x);
    for (auto& p : snap)
        if (p) cudaFree(p);
    if (st != GBP_OK) return st;
    if (e != cudaSuccess) return cuda_fail(g, e, "autotune");
    int best = -1;
    double best_mode[2] = {-1.0, -1.0};
    for (size_t c = 0; c < cand.size(); ++c) {
        if (ms[c] < 0) continue;
        if (best < 0 || ms[c] < ms[best]) best = (int)c;
        double& bm = best_mode[cand[c].first - 1];
        if (bm < 0 || ms[c] < bm) bm = ms[c];
    }
    if (best < 0) return fail(g, GBP_ECUDA, "autotune: no launch configuration ran");
    g->tuned_mode = cand[best].first;
    // each mode keeps its own best shape (launch_mode may force the other)
    for (size_t c = 0; c < cand.size(); ++c) {
        if (ms[c] < 0 || ms[c] != best_mode[cand[c].first - 1]) continue;
        if (cand[c].first == 1 && g->tuned_pshape < 0) g->tuned_pshape = cand[c].second;
        if (cand[c].first == 2 && g->tuned_fshape < 0) g->tuned_fshape = cand[c].second;
    }
    if (!tunable(g)) g->tuned_fshape = g->tuned_pshape = 0;
    gbp_tuning& T = g->tuning;
    T.n_candidates = (int32_t)std::min<size_t>(cand.size(), GBP_MAX_TUNING_CANDIDATES);
    for (int c = 0; c < T.n_candidates; ++c) {
        T.cand_mode[c] = cand[c].first;
        T.cand_shape[c] = cand[c].second;
        T.cand_ms[c] = ms[c];
    }
    tune_cache_store(g);
    if (chosen) *chosen = g->tuned_mode;
    if (ms_out) {
        ms_out[0] = best_mode[0];
        ms_out[1] = best_mode[1];
    }
    return GBP_OK;
}

gbp_status gbp_get_tuning(const gbp_graph* g, gbp_tuning* out) {
    if (!g || !out) return GBP_EINVAL;
    static const int f_threads[N_FACTOR_SHAPES] = {128, 128, 128, 64, 128, 128};
    static const int f_minb[N_FACTOR_SHAPES] = {1, 3, 4, 1, 4, 3};
    static const int p_minb[N_PERSISTENT_SHAPES] = {1};
    *out = g->tuning;
    out->launch_mode = g->prm.launch_mode ? g->prm.launch_mode : g->tuned_mode;
    out->factor_shape = factor_shape(g);
    out->persistent_shape = persistent_shape(g);
    out->factor_threads = f_threads[out->factor_shape];
    out->factor_min_blocks = f_minb[out->factor_shape];
    out->persistent_min_blocks = p_minb[out->persistent_shape];
    out->tile_factors = 32;
    return GBP_OK;
}

gbp_status gbp_add_keyframe(gbp_graph* g, const double* kf_Rt_init, int32_t n_new_lm, const double* new_lm_xyz,
                            int32_t n_obs, const int32_t* obs_lm, const double* obs_uv, int32_t* new_kf_index) {
    if (!g) return GBP_EINVAL;
    if (new_kf_index) *new_kf_index = -1;
    if (n_new_lm < 0 || n_obs < 0 || (n_obs && (!obs_lm || !obs_uv))) return fail(g, GBP_EINVAL, "bad counts");
    if (g->prob_kf0.size() != 2) return fail(g, GBP_ESTATE, "gbp_add_keyframe needs a single-problem graph");
    if (!kf_Rt_init && g->n_kf == 0) return fail(g, GBP_EINVAL, "no keyframe to copy the initial pose from");
    if (kf_Rt_init && !finite_all(kf_Rt_init, 12)) return fail(g, GBP_EINVAL, "initial pose not finite");
    if (new_lm_xyz && !finite_all(new_lm_xyz, 3 * (size_t)n_new_lm)) return fail(g, GBP_EINVAL, "points not finite");
    if (!finite_all(obs_uv, 2 * (size_t)n_obs)) return fail(g, GBP_EINVAL, "pixels not finite");
    const int L1 = g->n_lm + n_new_lm;
    std::vector<char> seen(n_new_lm, 0);
    for (int i = 0; i < n_obs; ++i) {
        if (obs_lm[i] < 0 || obs_lm[i] >= L1) return fail(g, GBP_EINVAL, "observation index out of range");
        if (obs_lm[i] >= g->n_lm) seen[obs_lm[i] - g->n_lm] = 1;
    }
    if (!new_lm_xyz)
        for (char c : seen)
            if (!c) return fail(g, GBP_EINVAL, "a new point without observation needs an initial position");
    gbp_status st = ensure_built(g);
    if (st != GBP_OK) return st;
    st = g->storage ? add_keyframe_impl<double>(g, kf_Rt_init, n_new_lm, new_lm_xyz, n_obs, obs_lm, obs_uv)
                    : add_keyframe_impl<float>(g, kf_Rt_init, n_new_lm, new_lm_xyz, n_obs, obs_lm, obs_uv);
    if (st == GBP_OK && new_kf_index) *new_kf_index = g->n_kf - 1;
    return st;
}

gbp_status gbp_set_partition(gbp_graph* g, int32_t kf_begin, int32_t kf_end, int32_t lm_begin, int32_t lm_end) {
    if (!g) return GBP_EINVAL;
    if (g->prob_kf0.size() != 2) return fail(g, GBP_ESTATE, "partitions apply to a single-problem graph");
    if (g->prm.precision_mode == 2) return fail(g, GBP_ESTATE, "partitions run the FP32 path");
    if (lm_end < 0) {   // back to the whole graph
        g->part_lm1 = -1;
    } else {
        if (kf_begin < 0 || kf_begin > kf_end || kf_end > g->n_kf || lm_begin < 0 || lm_begin > lm_end ||
            lm_end > g->n_lm)
            return fail(g, GBP_EINVAL, "partition range out of bounds");
        g->part_kf0 = kf_begin;
        g->part_kf1 = kf_end;
        g->part_lm0 = lm_begin;
        g->part_lm1 = lm_end;
    }
    destroy_exec(g);
    g->built = false;   // the tiles break at the landmark range: rebuilt, and reset to iteration 0
    return ensure_built(g);
}

gbp_status gbp_split_phase(gbp_graph* g, int32_t phase) {
    if (!g || phase < 0 || phase > 1) return GBP_EINVAL;
    if (g->part_lm1 < 0) return fail(g, GBP_ESTATE, "gbp_split_phase needs gbp_set_partition");
    if (g->prm.damping_mode != 0) return fail(g, GBP_ESTATE, "a partitioned graph runs the fixed damping schedule");
    gbp_status st = ensure_built(g);
    if (st != GBP_OK) return st;
    (void)cudaGetLastError();
    const DevGraph<float>& d = g->sf.g;
    const KParams<float> kp = make_kparams<float>(g);
    CK(phase == 0 ? launch_factor<float>(d, kp, g->stream, DAMP_FIXED, false, factor_shape(g))
                  : launch_belief<float>(d, kp, g->stream, false));
    g->launches += 1;
    g->last_mode = 2;
    return GBP_OK;
}

namespace {
gbp_status split_records(gbp_graph* g, int32_t kind, int32_t n, const int32_t* index, float* io, bool put) {
    if (!g || (kind != 0 && kind != 1) || n < 0 || (n && (!index || !io))) return GBP_EINVAL;
    if (g->storage != 0) return fail(g, GBP_ESTATE, "split records are FP32");
    if (n == 0) return GBP_OK;
    std::vector<int32_t> idx(n);
    for (int i = 0; i < n; ++i) {
        const int32_t v = index[i];
        if (kind == 0) {
            if (v < 0 || v >= g->n_f) return fail(g, GBP_EINVAL, "observation index out of range");
            idx[i] = g->f_of_obs[v];
        } else {
            if (v < 0 || v >= g->n_kf) return fail(g, GBP_EINVAL, "keyframe index out of range");
            idx[i] = v;
        }
    }
    const size_t width = kind == 0 ? (size_t)GBP_SPLIT_MSG_FLOATS : (size_t)GBP_SPLIT_KF_FLOATS;
    int32_t* d_idx = nullptr;
    float* d_io = nullptr;
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&d_idx), sizeof(int32_t) * n);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&d_io), sizeof(float) * width * n);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_idx, idx.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, g->stream);
    if (e == cudaSuccess && put) e = cudaMemcpyAsync(d_io, io, sizeof(float) * width * n, cudaMemcpyHostToDevice, g->stream);
    if (e == cudaSuccess) e = launch_split_records<float>(g->sf.g, kind, put ? 1 : 0, n, d_idx, d_io, g->stream);
    if (e == cudaSuccess && !put) e = cudaMemcpyAsync(io, d_io, sizeof(float) * width * n, cudaMemcpyDeviceToHost, g->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    if (d_idx) cudaFree(d_idx);
    if (d_io) cudaFree(d_io);
    if (e != cudaSuccess) return cuda_fail(g, e, "split records");
    return GBP_OK;
}
}  // namespace

gbp_status gbp_get_split_records(const gbp_graph* g, int32_t kind, int32_t n, const int32_t* index, float* out) {
    return split_records(const_cast<gbp_graph*>(g), kind, n, index, out, false);
}

gbp_status gbp_put_split_records(gbp_graph* g, int32_t kind, int32_t n, const int32_t* index, const float* in) {
    return split_records(g, kind, n, index, const_cast<float*>(in), true);
}

void gbp_destroy_graph(gbp_graph* g) {
    if (!g) return;
    destroy_exec(g);
    g->sf.release(&g->pool);
    g->sd.release(&g->pool);
    g->pool.clear();
    if (g->ctl) cudaFree(g->ctl);
    if (g->partials) cudaFree(g->partials);
    if (g->met) cudaFree(g->met);
    if (g->d_prob_f0) cudaFree(g->d_prob_f0);
    if (g->h_ctl) cudaFreeHost(g->h_ctl);
    if (g->h_met) cudaFreeHost(g->h_met);
    if (g->capture) cudaStreamDestroy(g->capture);
    if (g->mlp_frag) cudaFree(g->mlp_frag);
    if (g->mlp_bias) cudaFree(g->mlp_bias);
    delete g;
}

gbp_status gbp_set_damping_model(gbp_graph* g, const gbp_mlp* net) {
    if (!g) return GBP_EINVAL;
    if (!net) {
        g->has_model = false;
        return GBP_OK;
    }
    if (!g->mlp_frag) {
        destroy_exec(g);   // captured launches hold the (so far null) weight pointers
        CK(dev_alloc(&g->mlp_frag, FWD_FRAG_WORDS));
        CK(dev_alloc(&g->mlp_bias, MLP_BIAS_WORDS));
    }
    CK(mlp_copy_packed(net, g->mlp_frag, g->mlp_bias, g->stream));
    CK(cudaStreamSynchronize(g->stream));
    g->has_model = true;
    return GBP_OK;
}

gbp_status gbp_get_factor_order(const gbp_graph* g, int32_t* obs_index) {
    if (!g || (g->n_f && !obs_index)) return GBP_EINVAL;
    std::copy(g->obs_index.begin(), g->obs_index.end(), obs_index);
    return GBP_OK;
}

gbp_status gbp_capture_messages(gbp_graph* g) {
    if (!g) return GBP_EINVAL;
    gbp_status st = ensure_built(g);
    if (st != GBP_OK) return st;
    st = read_ctl(g);
    if (st != GBP_OK) return st;
    const int t = g->h_ctl[CTL_ITER];
    const size_t n = 9 * (size_t)std::max(g->n_f, 1);
    if (g->storage) {
        if (!g->sd.eta_inf) CK(dev_alloc(&g->sd.eta_inf, n));
        CK(launch_capture_messages<double>(g->sd.g, t, g->sd.eta_inf, g->stream));
    } else {
        if (!g->sf.eta_inf) CK(dev_alloc(&g->sf.eta_inf, n));
        CK(launch_capture_messages<float>(g->sf.g, t, g->sf.eta_inf, g->stream));
    }
    g->launches += 1;
    CK(cudaStreamSynchronize(g->stream));
    return GBP_OK;
}

gbp_status gbp_record_iterations(gbp_graph* g, int32_t n_iters, float* X, float* target) {
    if (!g || n_iters < 0) return GBP_EINVAL;
    if (n_iters > 0 && g->n_f > 0 && (!X || !target)) return GBP_EINVAL;
    if (reinterpret_cast<uintptr_t>(X) % 16 != 0) return fail(g, GBP_EINVAL, "X must be 16-byte aligned");
    gbp_status st = ensure_built(g);
    if (st != GBP_OK) return st;
    if (!(g->storage ? (void*)g->sd.eta_inf : (void*)g->sf.eta_inf))
        return fail(g, GBP_ESTATE, "no reference messages: call gbp_capture_messages first");
    st = g->storage ? record_iterations<double>(g, n_iters, X, target) : record_iterations<float>(g, n_iters, X, target);
    if (st != GBP_OK) return st;
    return read_ctl(g);
}

}  // extern "C"
