// Host engine of the C ABI declared in include/helm.h.
//
// An Engine advances a set of independent instances of one kernel class (dimension D,
// inner precision) together: every launch of an outer step covers all of its active
// instances (work items (instance, level) for the multigrid kernels, (instance, tile)
// for the residual), and instances that have finished are skipped on the device by
// their status word.  One outer step is captured once into the body of a CUDA graph
// WHILE node; the convergence kernel at the end of the body sets the loop condition,
// so a whole solve runs as a single graph launch with no host round trip per step.
//
// A helm_plan owns one Engine with a single instance (helm_solve); a helm_batch owns
// one Engine per kernel class and admits / retires instances between calls
// (continuous batching for the served stream).
#include "../../include/helm.h"
#include "launch.h"

#include <algorithm>
#include <atomic>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <vector>

using namespace helm;

namespace {

std::atomic<uint64_t> g_launches{0};
thread_local char g_errbuf[256] = "";
// engines launched on streams of decreasing priority by predicted work (else all equal)
constexpr bool g_lane_priority = true;

double lambda_min_of(int D, int n, double h);

// Predicted work of a solve: its outer steps from the closed-form contraction
// rho = |alpha + i p| / (lambda_min + sigma) (alpha = k^2 + sigma) and the tolerance, times n^D
double predicted_work(int D, int n, double h, double k2, double sigma, double damp, double tol, int max_outer)
{
    const double l = lambda_min_of(D, n, h);
    const double rho = std::hypot(k2 + sigma, damp) / (l + sigma);
    double steps = max_outer;
    if (rho > 0.0 && rho < 1.0 && tol > 0.0 && tol < 1.0) steps = std::min(steps, std::log(tol) / std::log(rho));
    return steps * std::pow((double)n, D);
}

#define HELM_CK(call)                                                                     \
    do {                                                                                  \
        cudaError_t _e = (call);                                                          \
        if (_e != cudaSuccess) {                                                          \
            snprintf(g_errbuf, sizeof g_errbuf, "%s: %s (%s:%d)", #call,                  \
                     cudaGetErrorString(_e), __FILE__, __LINE__);                         \
            return HELM_ECUDA;                                                            \
        }                                                                                 \
    } while (0)

int tail_n(int D, int prec) { return tail_top(D, prec == HELM_PREC_FP64); }
int elem_bytes(int prec) { return prec == HELM_PREC_FP64 ? 16 : 8; }
size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

bool is_pow2m1(int n) { return n >= 1 && ((n + 1) & n) == 0; }

int res_rows_per_tile(int D) { return residual_tile_rows(D); }
// residual tiles along z: 3D tiles march over residual_tile_planes(3) planes; 2D has one
int res_tz(int D, int n) { return D == 3 ? (n + residual_tile_planes(3) - 1) / residual_tile_planes(3) : 1; }

// Fill the geometry part of a descriptor and return the workspace bytes it needs (the
// level arrays, the second iterate buffer and the residual partials).  With base != NULL
// the pointers are carved out of it.
size_t layout(InstDesc& d, int D, int n, double h, double k, int prec, char* base)
{
    d.D = D;
    d.n = n;
    d.h = h;
    d.k2 = k * k;
    d.ih2 = 1.0 / (h * h);
    d.cdiag = d.k2 - 2.0 * D * d.ih2;
    d.damp = 0.0;
    int nl = 0, lt = -1;
    for (int m = n; m >= 1 && nl < HELM_MAXLEV; m = (m - 1) / 2) {
        if (lt < 0 && m <= tail_n(D, prec)) lt = nl;
        d.lev[nl].n = m;
        ++nl;
    }
    d.nlev = nl;
    d.ltail = lt;
    size_t off = 0;
    const size_t eb = elem_bytes(prec);
    double hl = h;
    for (int l = 0; l < nl; ++l) {
        LevelDesc& L = d.lev[l];
        L.h = hl;
        hl *= 2.0;
        L.rows = L.n + 2;
        L.pitch = round_up(L.n + 2, 16);
        L.e = nullptr;
        L.rhs = nullptr;
        L.e2 = nullptr;
        L.rhs2 = nullptr;
        if (l > lt) continue;               // deeper levels live only inside the tail kernel
        const size_t planes = (D == 3) ? (size_t)L.rows : 1;
        const size_t sz = align256((size_t)L.pitch * L.rows * planes * eb);
        const bool two = (D == 2 && l < lt);  // fused 2D levels keep a second iterate
        const bool r2 = two && l == 0;        // ... and level 0 a second right-hand side
        if (base) {
            L.e = base + off;
            L.rhs = base + off + sz;
            if (two) L.e2 = base + off + 2 * sz;
            if (r2) L.rhs2 = base + off + 3 * sz;
        }
        off += (two ? (r2 ? 4 : 3) : 2) * sz;
    }
    const size_t S = (size_t)n + 2;
    const size_t ubytes = align256(((D == 3) ? S * S * S : S * S) * 16);
    if (base) d.u[1] = (double2*)(base + off);
    off += ubytes;
    d.res_tx = (n + 31) / 32;
    d.res_ty = (n + res_rows_per_tile(D) - 1) / res_rows_per_tile(D);
    d.nres_blocks = d.res_tx * d.res_ty * res_tz(D, n);
    if (base) d.part = (double*)(base + off);
    off += align256((size_t)2 * d.nres_blocks * sizeof(double));
    if (base) d.count = (unsigned int*)(base + off);
    off += 256;
    set_shift(d, 0.0);
    return off;
}

// bytes of the level arrays to clear at allocation (rings must be zero)
struct Instance {
    InstDesc d{};
    int prec = 1;
    char* ws = nullptr;          // workspace (levels, u[1], partials)
    size_t ws_bytes = 0;
    double* hist = nullptr;      // device: relres (cap + 1) then einf (cap)
    int hist_cap = -1;
    bool hist_sep = false;       // hist has its own allocation (regrown by a longer solve)
    bool stream_ordered = false; // allocated with cudaMallocAsync
    ResItem* d_res0 = nullptr;   // this instance's residual tiles (initial residual)
    int nres0 = 0;
    char* io = nullptr;          // library-owned f, g, u (solves submitted from host memory)
    size_t io_bytes = 0;
    cudaEvent_t ready = nullptr; // their upload done (waited for before the solve starts)
};

struct LaunchRec {
    // UPRES1 names, in helm_batch_profile only, an UPRES launch that also forms level 1's
    // ascent (color 1); steps hold it as UPRES
    enum Kind { RBGS, RESTRICT, PROLONG, ZERO, TAIL, RESID, CHECK, DOWN, UP, UPRES, CTAIL, DOWN2, UPRES1, NKINDS } kind;
    int off, cnt, work, color, mode;
    double bytes;   // algorithmic bytes of one launch (each datum it must touch, once)
    int nmax = 0;   // DOWN: the largest level of the launch; UPRES: the level-0 size
    int ninst = 0;  // UPRES: instances of the launch (folded step control)
};

// The launch plan of one slot geometry: its work-item tables, launch sequences and the
// captured graph of one outer step (kernel parameters point into d_mg / d_res).
struct PlanState {
    std::vector<LaunchRec> step, vcyc_plain;
    std::vector<MgItem> h_items;
    MgItem* d_mg = nullptr;
    size_t mg_cap = 0;
    ResItem* d_res = nullptr;
    size_t res_cap = 0;
    int nres = 0, max_tail = 1, damp_any = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphConditionalHandle cond = 0;
    std::vector<long> plan_sig, graph_sig;

    void destroy()
    {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (d_mg) cudaFree(d_mg);
        if (d_res) cudaFree(d_res);
        exec = nullptr;
        graph = nullptr;
        d_mg = nullptr;
        d_res = nullptr;
        mg_cap = res_cap = 0;
    }
};

struct Engine {
    int D = 2, prec = 1;
    int nu1 = 2, nu2 = 2, cycles = 1;
    // 2D tile shape of the fused level kernels: HELM_TILES_AUTO (64 x 32, or 32 x 16 where
    // the large tiles would leave the GPU under-filled), _LARGE (64 x 32 wherever allowed),
    // _SMALL (32 x 16 on levels up to 511)
    int tiles = HELM_TILES_AUTO;
    // coarse levels of 2D complex64 cycles without pre-smoothing: HELM_COARSE_AUTO (levels
    // 255 and below in one 8-CTA cluster per instance when every instance is at least 511
    // and their clusters are resident at once), _CTA (one-CTA tail from level 63), _CLUSTER (the
    // cluster wherever it applies, and level 1's ascent inside the fused finest kernel: the
    // lowest latency for a solve alone, more work per step when solves share the GPU)
    int coarse = HELM_COARSE_AUTO;
    // With HELM_COARSE_AUTO, whether this engine is the caller's critical path: a plan's own
    // solve, or a batch's highest-priority lane holding a single solve.  Such an engine
    // forms level 1's ascent inside the fused finest kernel (as HELM_COARSE_CLUSTER does),
    // trading throughput it does not need for latency.
    bool latency = false;
    cudaStream_t cap_stream = nullptr;
    int cap = 0;                               // descriptor slots
    std::vector<Instance*> slots;              // nullptr = free
    InstDesc* d_desc = nullptr;
    InstState* d_state = nullptr;
    int* d_ctrl = nullptr;                     // [0] steps done, [1] step budget, [2] go, [3] arrivals
    int* h_ctrl = nullptr;                     // pinned mirror
    InstState* h_state = nullptr;              // pinned mirror (cap entries)
    // page-locked staging of a starting instance's descriptor and state (a copy from
    // pageable memory would wait for the stream; a slot is restaged only after its previous
    // instance retired, behind a stream synchronisation)
    InstDesc* h_desc_stage = nullptr;
    InstState* h_state_stage = nullptr;
    // the starts of the solves submitted since the last step, one launch of each kind for
    // all of them: their slots (page-locked staging, device copy) and residual tiles
    int* h_start_slots = nullptr;
    int* d_start_slots = nullptr;
    size_t start_cap = 0;
    ResItem* d_start_items = nullptr;
    size_t start_items_cap = 0;
    MgItem* d_mg = nullptr;
    size_t mg_cap = 0;
    ResItem* d_res = nullptr;
    size_t res_cap = 0;
    int nres = 0;
    std::vector<LaunchRec> step;               // one outer step
    std::vector<long> plan_sig;                // slot geometry the launch plan was built for
    std::vector<long> graph_sig;               // slot geometry the graph was captured for
    std::vector<MgItem> h_items;               // host copy of the multigrid work items
    std::vector<LaunchRec> vcyc_plain;         // one V-cycle from the current iterate
    int max_tail = 1;
    int damp_any = 0;                          // some slot's instance has p != 0
    bool dirty = true;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphConditionalHandle cond = 0;

    // Plans of other slot geometries, least recently used first: a batch whose geometry
    // alternates (solves joining a running batch, then retiring) reuses their graphs.
    static constexpr size_t PARKED_MAX = 3;
    std::vector<PlanState> parked;

    ~Engine() { release(); }

    void swap_plan(PlanState& p)
    {
        std::swap(step, p.step);
        std::swap(vcyc_plain, p.vcyc_plain);
        std::swap(h_items, p.h_items);
        std::swap(d_mg, p.d_mg);
        std::swap(mg_cap, p.mg_cap);
        std::swap(d_res, p.d_res);
        std::swap(res_cap, p.res_cap);
        std::swap(nres, p.nres);
        std::swap(max_tail, p.max_tail);
        std::swap(damp_any, p.damp_any);
        std::swap(graph, p.graph);
        std::swap(exec, p.exec);
        std::swap(cond, p.cond);
        std::swap(plan_sig, p.plan_sig);
        std::swap(graph_sig, p.graph_sig);
    }

    void release()
    {
        for (PlanState& p : parked) p.destroy();
        parked.clear();
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        exec = nullptr;
        graph = nullptr;
        if (d_desc) cudaFree(d_desc);
        if (d_state) cudaFree(d_state);
        if (d_ctrl) cudaFree(d_ctrl);
        if (h_ctrl) cudaFreeHost(h_ctrl);
        if (h_state) cudaFreeHost(h_state);
        if (h_desc_stage) cudaFreeHost(h_desc_stage);
        if (h_state_stage) cudaFreeHost(h_state_stage);
        if (h_start_slots) cudaFreeHost(h_start_slots);
        if (d_start_slots) cudaFree(d_start_slots);
        if (d_start_items) cudaFree(d_start_items);
        if (d_mg) cudaFree(d_mg);
        if (d_res) cudaFree(d_res);
        if (cap_stream) cudaStreamDestroy(cap_stream);
        d_desc = nullptr; d_state = nullptr; d_ctrl = nullptr; h_ctrl = nullptr;
        h_state = nullptr; d_mg = nullptr; d_res = nullptr; cap_stream = nullptr;
        h_desc_stage = nullptr; h_state_stage = nullptr;
        h_start_slots = nullptr; d_start_slots = nullptr; d_start_items = nullptr;
        start_cap = 0; start_items_cap = 0;
    }

    helm_status init(int D_, int prec_)
    {
        D = D_;
        prec = prec_;
        HELM_CK(cudaStreamCreateWithFlags(&cap_stream, cudaStreamNonBlocking));
        HELM_CK(cudaMalloc(&d_ctrl, 4 * sizeof(int)));
        HELM_CK(cudaMallocHost(&h_ctrl, 4 * sizeof(int)));
        HELM_CK(setup_tail(D, prec == HELM_PREC_FP64 ? 0 : 1));
        if (D == 2) HELM_CK(setup_2d(prec == HELM_PREC_FP64 ? 0 : 1));
        if (D == 2 && prec != HELM_PREC_FP64) ctail_setup();
        HELM_CK(setup_generic(D, prec == HELM_PREC_FP64 ? 0 : 1));
        HELM_CK(setup_outer());
        return grow(4);
    }

    helm_status grow(int want)
    {
        if (want <= cap) return HELM_OK;
        int nc = std::max(want, cap * 2);
        InstDesc* nd = nullptr;
        InstState* ns = nullptr;
        InstState* nh = nullptr;
        HELM_CK(cudaMalloc(&nd, sizeof(InstDesc) * nc));
        HELM_CK(cudaMalloc(&ns, sizeof(InstState) * nc));
        HELM_CK(cudaMallocHost(&nh, sizeof(InstState) * nc));
        InstDesc* hd = nullptr;
        InstState* hs = nullptr;
        HELM_CK(cudaMallocHost(&hd, sizeof(InstDesc) * nc));
        HELM_CK(cudaMallocHost(&hs, sizeof(InstState) * nc));
        std::vector<InstState> idle(nc);
        for (auto& s : idle) { memset(&s, 0, sizeof s); s.status = HELM_ST_IDLE; }
        if (cap > 0) {
            HELM_CK(cudaMemcpy(nd, d_desc, sizeof(InstDesc) * cap, cudaMemcpyDeviceToDevice));
            HELM_CK(cudaMemcpy(idle.data(), d_state, sizeof(InstState) * cap, cudaMemcpyDeviceToHost));
        }
        HELM_CK(cudaMemcpy(ns, idle.data(), sizeof(InstState) * nc, cudaMemcpyHostToDevice));
        if (d_desc) cudaFree(d_desc);
        if (d_state) cudaFree(d_state);
        if (h_state) cudaFreeHost(h_state);
        if (h_desc_stage) {
            // the old staging may still feed queued copies of earlier starts
            HELM_CK(cudaDeviceSynchronize());
            cudaFreeHost(h_desc_stage);
        }
        if (h_state_stage) cudaFreeHost(h_state_stage);
        d_desc = nd;
        d_state = ns;
        h_state = nh;
        h_desc_stage = hd;
        h_state_stage = hs;
        slots.resize(nc, nullptr);
        cap = nc;
        dirty = true;
        return HELM_OK;
    }

    // Rebuild the work-item lists and the launch sequence of one outer step for the
    // instances currently in the slots.
    helm_status rebuild_plan()
    {
        std::vector<MgItem> items;
        std::vector<ResItem> res;
        int J = 0;
        max_tail = 1;
        for (int i = 0; i < cap; ++i)
            if (slots[i]) {
                J = std::max(J, slots[i]->d.ltail);
                max_tail = std::max(max_tail, slots[i]->d.lev[slots[i]->d.ltail].n);
            }
        struct Ph { int off, cnt, w_rb, w_rs, w_pr, w_z; double b_rb, b_rs, b_pr, b_z; int tiles, shape, nmax; };
        const double eb = elem_bytes(prec);
        auto pts = [&](int m) { return (D == 3) ? (double)m * m * m : (double)m * m; };
        std::vector<Ph> ph(J);
        for (int j = 0; j < J; ++j) {
            Ph p{(int)items.size(), 0, 0, 0, 0, 0, 0.0, 0.0, 0.0, 0.0, 0, 0, 0};
            for (int i = 0; i < cap; ++i) {
                if (!slots[i]) continue;
                const InstDesc& d = slots[i]->d;
                const int l = j - (J - d.ltail);
                if (l < 0) continue;
                items.push_back(MgItem{i, l});
                const int n = d.lev[l].n, nc = d.lev[l + 1].n;
                const long rows = (D == 3) ? (long)n * n : n;
                p.w_rb = (int)std::max<long>(p.w_rb, rows * ((n + 1) / 2));
                p.w_rs = (int)std::max<long>(p.w_rs, (D == 3) ? (long)nc * nc * nc : (long)nc * nc);
                p.w_pr = (int)std::max<long>(p.w_pr, (D == 3) ? (long)n * n * n : (long)n * n);
                const long pz = (long)d.lev[l].pitch * d.lev[l].rows * ((D == 3) ? d.lev[l].rows : 1);
                p.w_z = (int)std::max<long>(p.w_z, pz);
                // half-sweep: this colour's rhs and new values, the other colour's iterate
                p.b_rb += 1.5 * pts(n) * eb;
                // restriction: fine e and rhs in, coarse rhs and zeroed coarse e out
                p.b_rs += (2.0 * pts(n) + 2.0 * pts(nc)) * eb;
                // prolongation: coarse e in, fine e in and out
                p.b_pr += (pts(nc) + 2.0 * pts(n)) * eb;
                p.b_z += pts(n) * eb;
                p.nmax = std::max(p.nmax, n);
                ++p.cnt;
            }
            // one tile shape per launch (that of its largest level) and the matching grid
            if (D == 2) {
                // small tiles only where the large ones would leave the GPU under-filled
                if (tiles == HELM_TILES_LARGE) p.shape = 0;
                else if (tiles == HELM_TILES_SMALL) p.shape = tile_shape2d(p.nmax);
                else p.shape = (tile_shape2d(p.nmax) == 1 && p.cnt * tiles2d_for(p.nmax, 0) < 2 * 152) ? 1 : 0;
                for (int q = p.off; q < p.off + p.cnt; ++q)
                    p.tiles = std::max(p.tiles, tiles2d_for(slots[items[q].inst]->d.lev[items[q].level].n, p.shape));
            }
            ph[j] = p;
        }
        // tail items grouped by their top size (one launch per size present)
        struct TailGroup { int off, cnt, n0; double bytes; };
        std::vector<TailGroup> tails;
        double b_l0 = 0.0, b_res = 0.0;
        for (int n0 = 1; n0 <= 63; n0 = 2 * n0 + 1) {
            TailGroup tg{(int)items.size(), 0, n0, 0.0};
            for (int i = 0; i < cap; ++i) {
                if (!slots[i]) continue;
                const InstDesc& d = slots[i]->d;
                if (d.lev[d.ltail].n != n0) continue;
                items.push_back(MgItem{i, d.ltail});
                ++tg.cnt;
                tg.bytes += 2.0 * pts(n0) * eb;                      // rhs in, e out
            }
            if (tg.cnt) tails.push_back(tg);
        }
        for (int i = 0; i < cap; ++i)
            if (slots[i]) {
                const InstDesc& d = slots[i]->d;
                b_l0 += pts(d.n) * eb;
                // residual + update: u, e, f in; u', r out
                b_res += pts(d.n) * (16.0 + eb + 16.0 + 16.0 + eb);
            }
        // level-0 items (zeroing when nu1 == 0)
        const int l0_off = (int)items.size();
        int nl0 = 0, w_l0 = 0;
        for (int i = 0; i < cap; ++i)
            if (slots[i]) {
                items.push_back(MgItem{i, 0});
                ++nl0;
                const LevelDesc& L = slots[i]->d.lev[0];
                w_l0 = std::max(w_l0, L.pitch * L.rows * ((D == 3) ? L.rows : 1));
            }
        for (int i = 0; i < cap; ++i) {
            if (!slots[i]) continue;
            const InstDesc& d = slots[i]->d;
            const int tz = res_tz(D, d.n);
            for (int z = 0; z < tz; ++z)
                for (int y = 0; y < d.res_ty; ++y)
                    for (int x = 0; x < d.res_tx; ++x) res.push_back(ResItem{i, x, y, z});
        }
        if (items.size() > mg_cap) {
            if (d_mg) cudaFree(d_mg);
            mg_cap = std::max(items.size(), mg_cap * 2);
            HELM_CK(cudaMalloc(&d_mg, mg_cap * sizeof(MgItem)));
        }
        if (res.size() > res_cap) {
            if (d_res) cudaFree(d_res);
            res_cap = std::max(res.size(), res_cap * 2);
            HELM_CK(cudaMalloc(&d_res, res_cap * sizeof(ResItem)));
        }
        h_items = items;
        if (!items.empty())
            HELM_CK(cudaMemcpy(d_mg, items.data(), items.size() * sizeof(MgItem), cudaMemcpyHostToDevice));
        if (!res.empty())
            HELM_CK(cudaMemcpy(d_res, res.data(), res.size() * sizeof(ResItem), cudaMemcpyHostToDevice));
        nres = (int)res.size();

        // cluster tail: every instance has a level 255 below its top (n >= 511), the cycle
        // has no pre-smoothing (every level it runs starts from zero) and nu2 <= 2
        bool use_ct = false;
        if (D == 2 && prec != HELM_PREC_FP64 && nu1 == 0 && (nu2 == 1 || nu2 == 2) &&
            coarse != HELM_COARSE_CTA && J >= 3) {
            int nocc = 0;
            bool all = true;
            for (int i = 0; i < cap; ++i) {
                if (!slots[i]) continue;
                const InstDesc& d = slots[i]->d;
                ++nocc;
                if (d.ltail < 3 || d.lev[d.ltail - 2].n != 255 || d.lev[d.ltail].n != 63) all = false;
            }
            const int maxc = ctail_setup();        // clusters resident at once
            use_ct = all && nocc > 0 && maxc > 0 && (coarse == HELM_COARSE_CLUSTER || nocc <= maxc);
        }
        auto tail = [&](std::vector<LaunchRec>& out, bool zero_start) {
            for (const TailGroup& tg : tails)
                out.push_back({LaunchRec::TAIL, tg.off, tg.cnt, tg.n0, 0, zero_start ? 0 : 1, tg.bytes});
        };
        auto vcycle2d = [&](std::vector<LaunchRec>& out, bool zero_start) {
            const int Jf = use_ct ? J - 2 : J;         // levels of the fused tile kernels
            // without pre-smoothing from a zero start every descent step restricts rhs alone:
            // two of them per launch, where every instance of the second phase is in the
            // first (no instance has its top level at the second)
            const bool pairs = nu1 == 0 && zero_start;
            for (int j = 0; j < Jf;) {
                if (pairs && j + 1 < Jf && ph[j + 1].cnt == ph[j].cnt) {
                    out.push_back({LaunchRec::DOWN2, ph[j].off, ph[j].cnt, 0, 0, 2, 0.0, ph[j].nmax});
                    j += 2;
                } else {
                    out.push_back({LaunchRec::DOWN, ph[j].off, ph[j].cnt, ph[j].tiles, ph[j].shape,
                                   zero_start ? 2 : 1, 0.0, ph[j].nmax});
                    j += 1;
                }
            }
            if (use_ct)
                out.push_back({LaunchRec::CTAIL, ph[Jf].off, ph[Jf].cnt, 0, 0, 0,
                               2.0 * pts(255) * eb * ph[Jf].cnt});
            else
                tail(out, zero_start);
            // without pre-smoothing the descent leaves e2 unwritten where the iterate was zero
            const int e2_mode = (nu1 == 0) ? (zero_start ? 2 : 1) : 0;
            for (int j = Jf - 1; j >= 0; --j)
                out.push_back({LaunchRec::UP, ph[j].off, ph[j].cnt, ph[j].tiles, ph[j].shape, e2_mode, 0.0});
        };
        auto vcycle = [&](std::vector<LaunchRec>& out, bool zero_start) {
            if (D == 2 && nu1 <= 4 && nu2 <= 4) { vcycle2d(out, zero_start); return; }
            // without pre-smoothing the iterates are zero on the way down (every level from a
            // zero start, the coarse ones otherwise): the restriction takes rhs alone and the
            // prolongation assigns
            const int zmode = (nu1 == 0) ? (zero_start ? 2 : 1) : 0;
            for (int j = 0; j < J; ++j) {
                for (int s = 0; s < nu1; ++s) {
                    const int mode = (s == 0) ? (zero_start ? 2 : 1) : 0;
                    out.push_back({LaunchRec::RBGS, ph[j].off, ph[j].cnt, ph[j].w_rb, 0, mode, ph[j].b_rb, ph[j].nmax});
                    out.push_back({LaunchRec::RBGS, ph[j].off, ph[j].cnt, ph[j].w_rb, 1, 0, ph[j].b_rb, ph[j].nmax});
                }
                out.push_back({LaunchRec::RESTRICT, ph[j].off, ph[j].cnt, ph[j].w_rs, 0, zmode, ph[j].b_rs, ph[j].nmax});
            }
            tail(out, zero_start);
            for (int j = J - 1; j >= 0; --j) {
                out.push_back({LaunchRec::PROLONG, ph[j].off, ph[j].cnt, ph[j].w_pr, 0, zmode, ph[j].b_pr});
                for (int s = 0; s < nu2; ++s) {
                    out.push_back({LaunchRec::RBGS, ph[j].off, ph[j].cnt, ph[j].w_rb, 0, 0, ph[j].b_rb, ph[j].nmax});
                    out.push_back({LaunchRec::RBGS, ph[j].off, ph[j].cnt, ph[j].w_rb, 1, 0, ph[j].b_rb, ph[j].nmax});
                }
            }
        };
        step.clear();
        for (int c = 0; c < cycles; ++c) vcycle(step, c == 0);
        // the residual launch also ends the step (its last instance to finish sets the
        // loop condition), so a step has no separate check launch
        int nocc = 0;
        damp_any = 0;
        for (int i = 0; i < cap; ++i) {
            nocc += slots[i] ? 1 : 0;
            if (slots[i] && slots[i]->d.damp != 0.0) damp_any = 1;
        }
        // 2D complex64 instances of one size whose level 0 is a fused level: level 0's final
        // ascent and the residual launch become one kernel (k_upres2d)
        bool fuse = D == 2 && prec != HELM_PREC_FP64 && nu1 <= 4 && nu2 <= 4 && J > 0 && nocc > 0 &&
                    !step.empty() && step.back().kind == LaunchRec::UP && step.back().off == ph[0].off &&
                    ph[0].cnt == nocc;
        int n_all = -1;
        for (int i = 0; i < cap && fuse; ++i) {
            if (!slots[i]) continue;
            const InstDesc& d = slots[i]->d;
            if ((n_all >= 0 && d.n != n_all) || d.ltail < 1 || !d.lev[0].rhs2) fuse = false;
            n_all = d.n;
        }
        if (fuse) {
            const int e2_mode = step.back().mode;
            // level 1's ascent inside the fused kernel too (its launch dropped): no
            // pre-smoothing (level 1's iterate and e2 zero), level 1 a fused level of every
            // instance, its ascent the launch right before
            const size_t m = step.size();
            const bool l1f = nu1 == 0 && J >= 2 && m >= 2 && step[m - 2].kind == LaunchRec::UP &&
                             step[m - 2].off == ph[1].off && ph[1].cnt == nocc &&
                             (coarse == HELM_COARSE_CLUSTER || (coarse == HELM_COARSE_AUTO && latency));
            step.back() = {LaunchRec::UPRES, ph[0].off, ph[0].cnt, upres2d_tiles(n_all), l1f ? 1 : 0, e2_mode,
                           0.0, n_all, nocc};
            if (l1f) step.erase(step.end() - 2);
        } else {
            step.push_back({LaunchRec::RESID, 0, nres, nocc, 1, 1, b_res});
        }
        vcyc_plain.clear();
        vcycle(vcyc_plain, false);
        return HELM_OK;
    }

    // Algorithmic bytes of one launch counting only the instances still iterating
    // (finished instances' blocks exit at once and move no data).
    double launch_bytes(const LaunchRec& L, const InstState* st) const
    {
        const double eb = elem_bytes(prec);
        auto pts = [&](int m) { return (D == 3) ? (double)m * m * m : (double)m * m; };
        double b = 0.0;
        if (L.kind == LaunchRec::RESID) {
            for (int i = 0; i < cap; ++i)
                if (slots[i] && st[i].status == HELM_ST_ACTIVE)
                    b += pts(slots[i]->d.n) * (16.0 + eb + 16.0 + 16.0 + eb);
            return b;
        }
        if (L.kind == LaunchRec::CHECK) return 0.0;
        if (L.kind == LaunchRec::UPRES) {
            // [e2], r_N, coarse e, u_N, f in; u_{N+1}, r_{N+1} out
            const bool e2z = (L.mode == 2);
            for (int i = 0; i < cap; ++i)
                if (slots[i] && st[i].status == HELM_ST_ACTIVE) {
                    const InstDesc& d = slots[i]->d;
                    b += pts(d.n) * ((e2z ? 1.0 : 2.0) * eb + 16.0 + 16.0 + 16.0 + eb) + pts(d.lev[1].n) * eb;
                    if (L.color) b += pts(d.lev[2].n) * eb;       // level 1 fused: its rhs, level 2's e
                }
            return b;
        }
        for (int q = L.off; q < L.off + L.cnt; ++q) {
            const MgItem& it = h_items[q];
            if (!slots[it.inst] || st[it.inst].status != HELM_ST_ACTIVE) continue;
            const InstDesc& d = slots[it.inst]->d;
            const int n = d.lev[it.level].n;
            const int nc = (it.level + 1 < d.nlev) ? d.lev[it.level + 1].n : 0;
            switch (L.kind) {
            case LaunchRec::RBGS: b += 1.5 * pts(n) * eb; break;
            case LaunchRec::RESTRICT: {
                const bool z = (L.mode == 2) || (L.mode == 1 && it.level > 0);
                b += (z ? (pts(n) + pts(nc)) : (2.0 * pts(n) + 2.0 * pts(nc))) * eb;
                break;
            }
            case LaunchRec::PROLONG: {
                const bool z = (L.mode == 2) || (L.mode == 1 && it.level > 0);
                b += (pts(nc) + (z ? 1.0 : 2.0) * pts(n)) * eb;
                break;
            }
            case LaunchRec::ZERO: b += pts(n) * eb; break;
            case LaunchRec::TAIL: b += 2.0 * pts(n) * eb; break;
            case LaunchRec::CTAIL: b += 2.0 * pts(n) * eb; break;
            case LaunchRec::DOWN2: b += (pts(n) + pts(nc) + pts((nc - 1) / 2)) * eb; break;
            case LaunchRec::DOWN: {
                const bool zero = (L.mode == 2) || (L.mode == 1 && it.level > 0);
                if (zero && nu1 == 0) b += (pts(n) + pts(nc)) * eb;      // rhs in, coarse rhs out
                else b += ((zero ? 2.0 : 3.0) * pts(n) + pts(nc)) * eb;  // [e], rhs in; e2, coarse rhs out
                break;
            }
            case LaunchRec::UP: {
                const bool e2z = (L.mode == 2) || (L.mode == 1 && it.level > 0);
                b += ((e2z ? 2.0 : 3.0) * pts(n) + pts(nc)) * eb;         // [e2], rhs, coarse e in; e out
                break;
            }
            default: break;
            }
        }
        return b;
    }

    helm_status enqueue(const std::vector<LaunchRec>& seq, cudaStream_t s, bool use_cond)
    {
        for (const LaunchRec& L : seq) {
            cudaError_t e = cudaSuccess;
            switch (L.kind) {
            case LaunchRec::RBGS:
                e = launch_rbgs(D, prec, d_desc, d_state, d_mg + L.off, L.cnt, L.work, L.color, L.mode, s, L.nmax);
                break;
            case LaunchRec::RESTRICT:
                e = launch_restrict(D, prec, d_desc, d_state, d_mg + L.off, L.cnt, L.work, s, L.mode, L.nmax);
                break;
            case LaunchRec::PROLONG:
                // the sweeps that follow start with colour 0
                e = launch_prolong(D, prec, d_desc, d_state, d_mg + L.off, L.cnt, L.work, s, L.mode,
                                   nu2 > 0 ? 1 : 0);
                break;
            case LaunchRec::ZERO:
                e = launch_zero(D, prec, d_desc, d_state, d_mg + L.off, L.cnt, L.work, s);
                break;
            case LaunchRec::TAIL:
                e = launch_tail(D, prec, L.work, d_desc, d_state, d_mg + L.off, L.cnt, nu1, nu2,
                                L.mode, s);
                break;
            case LaunchRec::CTAIL:
                e = launch_ctail(d_desc, d_state, d_mg + L.off, L.cnt, nu2, s);
                break;
            case LaunchRec::DOWN2:
                e = launch_restrict2_2d(prec, d_desc, d_state, d_mg + L.off, L.cnt, L.nmax, s);
                break;
            case LaunchRec::DOWN:
                e = launch_down2d(prec, d_desc, d_state, d_mg + L.off, L.cnt, L.work, nu1, L.mode, L.color, s,
                                  L.nmax);
                break;
            case LaunchRec::UP:
                e = launch_up2d(prec, d_desc, d_state, d_mg + L.off, L.cnt, L.work, nu2, L.color, L.mode, s);
                break;
            case LaunchRec::RESID:
                if (L.color)      // folded step control: L.work instances, cap statuses
                    e = launch_residual(D, prec, d_desc, d_state, d_res + L.off, L.cnt, L.mode, s,
                                        d_ctrl, cap, L.work, use_cond ? 1 : 0, (unsigned long long)cond,
                                        damp_any);
                else
                    e = launch_residual(D, prec, d_desc, d_state, d_res + L.off, L.cnt, L.mode, s,
                                        nullptr, 0, 0, 0, 0, damp_any);
                break;
            case LaunchRec::UPRES:     // color: level 1 fused
                e = launch_upres2d(d_desc, d_state, d_mg + L.off, L.cnt, L.nmax, nu2, L.mode, s, d_ctrl, cap,
                                   L.ninst, use_cond ? 1 : 0, (unsigned long long)cond, damp_any, L.color);
                break;
            case LaunchRec::CHECK:
                e = launch_check(d_state, L.cnt, d_ctrl, use_cond ? 1 : 0,
                                 (unsigned long long)cond, s);
                break;
            }
            if (e != cudaSuccess) {
                snprintf(g_errbuf, sizeof g_errbuf, "kernel launch: %s", cudaGetErrorString(e));
                return HELM_ECUDA;
            }
        }
        return HELM_OK;
    }

    // (Re)build the graph: a single WHILE node whose body is one outer step.
    helm_status build_graph()
    {
        if (exec) { cudaGraphExecDestroy(exec); exec = nullptr; }
        if (graph) { cudaGraphDestroy(graph); graph = nullptr; }
        HELM_CK(cudaGraphCreate(&graph, 0));
        HELM_CK(cudaGraphConditionalHandleCreate(&cond, graph, 1, cudaGraphCondAssignDefault));
        cudaGraphNodeParams p = {cudaGraphNodeTypeConditional};
        p.conditional.handle = cond;
        p.conditional.type = cudaGraphCondTypeWhile;
        p.conditional.size = 1;
        cudaGraphNode_t node;
        HELM_CK(cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &p));
        cudaGraph_t body = p.conditional.phGraph_out[0];
        HELM_CK(cudaStreamBeginCaptureToGraph(cap_stream, body, nullptr, nullptr, 0,
                                              cudaStreamCaptureModeThreadLocal));
        helm_status st = enqueue(step, cap_stream, true);
        cudaGraph_t captured = nullptr;
        cudaError_t e = cudaStreamEndCapture(cap_stream, &captured);
        if (st != HELM_OK) return st;
        HELM_CK(e);
        HELM_CK(cudaGraphInstantiate(&exec, graph, 0));
        return HELM_OK;
    }

    // What the launch plan and its graph depend on: the slot geometry, the cycle, and
    // whether any instance has a damping term (it selects the residual kernels' variant).
    std::vector<long> current_signature() const
    {
        std::vector<long> sig{cap, nu1, nu2, cycles, tiles, coarse, latency ? 1L : 0L};
        long damp = 0;
        for (int i = 0; i < cap; ++i) {
            sig.push_back(slots[i] ? (long)slots[i]->d.n * 4 + (long)slots[i]->d.D : -1L);
            if (slots[i] && slots[i]->d.damp != 0.0) damp = 1;
        }
        sig.push_back(damp);
        return sig;
    }

    // Make the launch plan (work items, launch sequence) match the slots.  The plan only
    // depends on the geometry of the occupied slots (pointers live in the device
    // descriptors), so re-admitting same-sized solves into the same slots keeps it.
    helm_status prepare_plan()
    {
        if (!dirty) return HELM_OK;
        std::vector<long> sig = current_signature();
        if (sig != plan_sig) {
            // park the current plan (a plan invalidated by a temporary rebuild is dropped)
            PlanState cur;
            swap_plan(cur);
            if (!cur.plan_sig.empty()) {
                parked.push_back(std::move(cur));
                if (parked.size() > PARKED_MAX) {
                    parked.front().destroy();
                    parked.erase(parked.begin());
                }
            } else {
                cur.destroy();
            }
            auto it = std::find_if(parked.begin(), parked.end(),
                                   [&](const PlanState& p) { return p.plan_sig == sig; });
            if (it != parked.end()) {
                swap_plan(*it);                 // the engine's fields were empty
                parked.erase(it);
            } else {
                helm_status st = rebuild_plan();
                if (st != HELM_OK) return st;
                plan_sig = sig;
            }
        }
        dirty = false;
        return HELM_OK;
    }

    bool graph_current() const { return exec != nullptr && graph_sig == plan_sig && !plan_sig.empty(); }

    // Plan and the CUDA graph of one outer step (re-captured when the plan changed).
    helm_status prepare()
    {
        helm_status st = prepare_plan();
        if (st != HELM_OK) return st;
        if (graph_current()) return HELM_OK;
        st = build_graph();
        if (st != HELM_OK) return st;
        graph_sig = plan_sig;
        return HELM_OK;
    }

    int active_count() const
    {
        int c = 0;
        for (auto* p : slots) c += p != nullptr;
        return c;
    }

    // the largest / the total predicted work of the active instances
    double longest_job() const
    {
        double w = 0.0;
        for (auto* p : slots)
            if (p) w = std::max(w, predicted_work(p->d.D, p->d.n, p->d.h, p->d.k2, p->d.sigma, p->d.damp, p->d.tol,
                                                   p->d.max_outer));
        return w;
    }
    double total_work() const
    {
        double w = 0.0;
        for (auto* p : slots)
            if (p) w += predicted_work(p->d.D, p->d.n, p->d.h, p->d.k2, p->d.sigma, p->d.damp, p->d.tol,
                                       p->d.max_outer);
        return w;
    }

    // Initial residual and norm of one newly started instance.
    // Batches start a submitted instance at its first step, on the stream its lane then
    // runs on, so the start kernels of the lanes run side by side.
    std::vector<int> pending;
    helm_status start_pending(cudaStream_t s)
    {
        std::vector<int> ps;
        for (int slot : pending)
            if (slot < cap && slots[slot]) ps.push_back(slot);
        pending.clear();
        std::sort(ps.begin(), ps.end());
        ps.erase(std::unique(ps.begin(), ps.end()), ps.end());
        bool one_size = true;
        for (int slot : ps) one_size = one_size && slots[slot]->d.n == slots[ps[0]]->d.n;
        if (ps.size() <= 1 || !one_size) {
            for (int slot : ps) {
                const helm_status st = start_instance(slot, s);
                if (st != HELM_OK) return st;
            }
            return HELM_OK;
        }
        // their uploads from host memory; descriptors and initial states, one copy per run
        // of consecutive slots
        for (int slot : ps)
            if (slots[slot]->ready) HELM_CK(cudaStreamWaitEvent(s, slots[slot]->ready, 0));
        for (int slot : ps) {
            InstState& init = h_state_stage[slot];
            memset(&init, 0, sizeof init);
            init.status = HELM_ST_ACTIVE;
            h_desc_stage[slot] = slots[slot]->d;
        }
        for (size_t i = 0; i < ps.size();) {
            size_t j = i + 1;
            while (j < ps.size() && ps[j] == ps[j - 1] + 1) ++j;
            const int a = ps[i], c = (int)(j - i);
            HELM_CK(cudaMemcpyAsync(d_desc + a, h_desc_stage + a, c * sizeof(InstDesc), cudaMemcpyHostToDevice, s));
            HELM_CK(cudaMemcpyAsync(d_state + a, h_state_stage + a, c * sizeof(InstState), cudaMemcpyHostToDevice,
                                    s));
            i = j;
        }
        // the slots, those without a damping term first (it selects the residual kernel's
        // variant, as for a single start)
        const int m = (int)ps.size();
        if ((size_t)m > start_cap) {
            if (h_start_slots) cudaFreeHost(h_start_slots);
            if (d_start_slots) cudaFree(d_start_slots);
            h_start_slots = nullptr;
            d_start_slots = nullptr;
            start_cap = 0;
            HELM_CK(cudaMallocHost(&h_start_slots, m * sizeof(int)));
            HELM_CK(cudaMalloc(&d_start_slots, m * sizeof(int)));
            start_cap = m;
        }
        int m0 = 0;
        for (int slot : ps)
            if (slots[slot]->d.damp == 0.0) h_start_slots[m0++] = slot;
        int q = m0;
        for (int slot : ps)
            if (slots[slot]->d.damp != 0.0) h_start_slots[q++] = slot;
        HELM_CK(cudaMemcpyAsync(d_start_slots, h_start_slots, m * sizeof(int), cudaMemcpyHostToDevice, s));
        const InstDesc& d0 = slots[ps[0]]->d;
        HELM_CK(launch_set_ring_many(D, d_desc, d_start_slots, m, d0.n, s));
        const int tx = d0.res_tx, ty = d0.res_ty, tz = res_tz(D, d0.n), T = tx * ty * tz;
        if ((size_t)m * T > start_items_cap) {
            if (d_start_items) cudaFree(d_start_items);
            d_start_items = nullptr;
            start_items_cap = 0;
            HELM_CK(cudaMalloc(&d_start_items, (size_t)m * T * sizeof(ResItem)));
            start_items_cap = (size_t)m * T;
        }
        HELM_CK(launch_fill_res_many(d_start_items, d_start_slots, m, tx, ty, tz, s));
        // the initial residuals; the last tile of each instance records its relres_0 and
        // initial status
        if (m0 > 0)
            HELM_CK(launch_residual(D, prec, d_desc, d_state, d_start_items, m0 * T, 0, s, nullptr, 0, 0, 0, 0, 0));
        if (m > m0)
            HELM_CK(launch_residual(D, prec, d_desc, d_state, d_start_items + (size_t)m0 * T, (m - m0) * T, 0, s,
                                    nullptr, 0, 0, 0, 0, 1));
        g_launches += 2 + (m0 > 0 ? 1 : 0) + (m > m0 ? 1 : 0);
        return HELM_OK;
    }

    helm_status start_instance(int slot, cudaStream_t s)
    {
        Instance* in = slots[slot];
        if (in->ready) HELM_CK(cudaStreamWaitEvent(s, in->ready, 0));   // its upload from host memory
        InstState& init = h_state_stage[slot];
        memset(&init, 0, sizeof init);
        init.status = HELM_ST_ACTIVE;
        h_desc_stage[slot] = in->d;
        HELM_CK(cudaMemcpyAsync(d_desc + slot, h_desc_stage + slot, sizeof(InstDesc), cudaMemcpyHostToDevice, s));
        HELM_CK(cudaMemcpyAsync(d_state + slot, &init, sizeof(InstState), cudaMemcpyHostToDevice, s));
        HELM_CK(launch_set_ring(D, d_desc, slot, in->d.n, s));
        // the instance's own tile list names instance 0: offset the tables to its slot;
        // the last tile records relres_0 and the initial status
        HELM_CK(launch_residual(D, prec, d_desc + slot, d_state + slot, in->d_res0, in->nres0, 0, s,
                                nullptr, 0, 0, 0, 0, in->d.damp != 0.0 ? 1 : 0));
        g_launches += 2;
        return HELM_OK;
    }

    // Run outer steps until every active instance has finished or `budget` steps ran.
    // Returns the number of steps executed (read back after the stream drains).
    helm_status run(cudaStream_t s, int budget, int* steps_done)
    {
        helm_status st = prepare();
        if (st != HELM_OK) return st;
        h_ctrl[0] = 0;
        h_ctrl[1] = budget > 0 ? budget : INT_MAX;
        h_ctrl[2] = 1;
        h_ctrl[3] = 0;
        HELM_CK(cudaMemcpyAsync(d_ctrl, h_ctrl, 4 * sizeof(int), cudaMemcpyHostToDevice, s));
        HELM_CK(cudaGraphLaunch(exec, s));
        HELM_CK(cudaMemcpyAsync(h_ctrl, d_ctrl, 3 * sizeof(int), cudaMemcpyDeviceToHost, s));
        HELM_CK(cudaMemcpyAsync(h_state, d_state, sizeof(InstState) * cap, cudaMemcpyDeviceToHost, s));
        HELM_CK(cudaStreamSynchronize(s));
        if (steps_done) *steps_done = h_ctrl[0];
        g_launches += (uint64_t)h_ctrl[0] * step.size();
        return HELM_OK;
    }
};

// One allocation per instance: the workspace (levels, u[1], partials), then its residual
// tile list, then the relres / increment histories.
// With `init`, the workspace's zeroing and tile list are left to the caller's batched
// set-up (launch_init_workspaces), described in *init; else done here on `s`.
helm_status alloc_instance(Instance& in, int D, int n, double h, double k, int prec,
                           int max_outer, cudaStream_t s, bool stream_ordered, size_t io_bytes = 0,
                           WsInit* init = nullptr)
{
    in.prec = prec;
    in.stream_ordered = stream_ordered;
    in.ws_bytes = layout(in.d, D, n, h, k, prec, nullptr);
    const int tz = res_tz(D, n);
    in.nres0 = tz * in.d.res_ty * in.d.res_tx;
    const size_t rb = align256((size_t)in.nres0 * sizeof(ResItem));
    in.hist_cap = max_outer;
    const size_t hb = (2 * (size_t)max_outer + 1) * sizeof(double);
    const size_t total = align256(in.ws_bytes) + rb + align256(hb) + io_bytes;
    if (stream_ordered) {
        HELM_CK(cudaMallocAsync((void**)&in.ws, total, s));
    } else {
        cudaError_t e = cudaMalloc((void**)&in.ws, total);
        if (e != cudaSuccess) {
            cudaGetLastError();
            snprintf(g_errbuf, sizeof g_errbuf, "cudaMalloc(%zu): %s", total, cudaGetErrorString(e));
            return HELM_ENOMEM;
        }
    }
    layout(in.d, D, n, h, k, prec, in.ws);
    // rings of the level iterates must be zero (everything is cleared once), and the
    // residual tiles of this instance (for its initial residual) are listed on the device
    in.d_res0 = (ResItem*)(in.ws + align256(in.ws_bytes));
    if (init) {
        *init = WsInit{(unsigned char*)in.ws, (unsigned long long)in.ws_bytes, in.d_res0, in.d.res_tx, in.d.res_ty,
                       tz, 0};
    } else {
        HELM_CK(cudaMemsetAsync(in.ws, 0, in.ws_bytes, s));
        HELM_CK(launch_fill_res_items(in.d_res0, in.d.res_tx, in.d.res_ty, tz, s));
        g_launches += 1;
    }
    in.hist = (double*)((char*)in.d_res0 + rb);
    in.d.hist = in.hist;
    in.d.einf = in.hist + max_outer + 1;
    in.io = io_bytes ? (char*)in.hist + align256(hb) : nullptr;
    in.io_bytes = io_bytes;
    return HELM_OK;
}

void free_instance(Instance& in, cudaStream_t s)
{
    if (in.ws) {
        if (in.stream_ordered) cudaFreeAsync(in.ws, s);
        else cudaFree(in.ws);
    }
    if (in.hist_sep && in.hist) cudaFree(in.hist);
    if (in.ready) cudaEventDestroy(in.ready);
    in.ready = nullptr;
    in.io = nullptr;
    in.hist_sep = false;
    in.ws = nullptr;
    in.d_res0 = nullptr;
    in.hist = nullptr;
}

helm_status check_ptr(const void* p)
{
    if (!p) return HELM_EINVAL;
    if (((uintptr_t)p & 15) != 0) return HELM_EINVAL;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return HELM_EINVAL;
    }
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged) return HELM_EINVAL;
    return HELM_OK;
}

bool overlap(const void* a, size_t na, const void* b, size_t nb)
{
    const char* x = (const char*)a;
    const char* y = (const char*)b;
    return x < y + nb && y < x + na;
}

double lambda_min_of(int D, int n, double h)
{
    const double pi = 3.14159265358979323846;
    const double s = std::sin(pi / (2.0 * (n + 1)));
    return D * 4.0 / (h * h) * s * s;
}

}  // namespace

struct helm_plan {
    int D, n, prec;
    double h, k;
    double alpha, damp;        // general cavity (Section 2.2): alpha >= k^2, p >= 0
    double sigma;              // alpha - k^2, computed once (0 exactly for alpha = k^2)
    cudaStream_t stream;
    Engine eng;
    Instance inst;
    size_t points() const { return D == 3 ? (size_t)n * n * n : (size_t)n * n; }
    size_t padded() const { size_t s = n + 2; return D == 3 ? s * s * s : s * s; }
};

struct helm_batch {
    size_t cap_bytes = 0, used = 0;
    int nu1 = 2, nu2 = 2, cycles = 1;           // inner schedule of every engine
    int tiles = HELM_TILES_AUTO;                // 2D tile-shape policy of every engine
    int coarse = HELM_COARSE_AUTO;              // coarse-level policy of every engine
    // per kernel class (2 D + prec): a schedule set by helm_batch_set_cycle_class, used
    // instead of the batch-wide one by that class's engines ({0, 0, 0}: none)
    int cls_sched[8][3] = {};
    // Solves of one kernel class are spread over `lanes` engines (each with its own graph
    // on its own stream, launched concurrently), so one lane's FP64-bound residual runs
    // beside another lane's latency-bound coarse levels.
    int lanes = 4;
    cudaStream_t stream = nullptr;
    // uploads of solves submitted from host memory (helm_batch_submit_host), in submission
    // order, so that the first solve starts while the others' data are still coming in
    cudaStream_t up_stream = nullptr;
    cudaEvent_t up_fork = nullptr;
    // key = engine_key(class 2 D + prec, grid-size group log2(n + 1), lane)
    std::map<int, std::unique_ptr<Engine>> engines;
    // A step launches the engines on streams of decreasing priority, ordered by their
    // longest predicted job, so the critical path's kernels are scheduled first and the
    // shorter solves fill the SMs it leaves idle.
    std::vector<cudaStream_t> rank_streams;
    std::vector<cudaEvent_t> rank_join;
    cudaEvent_t fork = nullptr;
    struct Rec {
        int key = 0, slot = -1;
        int done = 0, status = 0, iters = 0;
        Instance* inst = nullptr;
        void* u = nullptr;
        size_t ubytes = 0;
        std::vector<double> hist;
        void* host_u = nullptr;         // helm_batch_set_host_result: the result's host copy
        bool host_pinned = false;       // page-locked: copied behind the lane's last step
        bool host_sent = false;         // its copy was queued behind the lane's last step
    };
    std::map<uint64_t, Rec> recs;
    uint64_t next = 1;
    // page-locked staging of retiring solves' relres histories (one copy per solve, one
    // synchronisation for all of them)
    double* h_hist = nullptr;
    size_t h_hist_cap = 0;
    // workspaces of the solves submitted since the batch last ran: zeroed, and their tile
    // lists written, by one launch before its next step (records staged page-locked, then
    // copied to the device)
    std::vector<WsInit> init_pending;
    WsInit* h_init = nullptr;
    WsInit* d_init = nullptr;
    size_t init_cap = 0;
};

namespace helm {
// shared with the other translation units of the library (annulus.cu)
void note_error(const char* msg) { snprintf(g_errbuf, sizeof g_errbuf, "%s", msg); }
void add_launches(uint64_t n) { g_launches += n; }
bool device_pointer_ok(const void* p) { return check_ptr(p) == HELM_OK; }
}  // namespace helm

extern "C" {

const char* helm_status_str(int s)
{
    switch (s) {
    case HELM_CONVERGED: return "HELM_CONVERGED";
    case HELM_MAXITER: return "HELM_MAXITER";
    case HELM_DIVERGED: return "HELM_DIVERGED";
    case HELM_EINVAL: return "HELM_EINVAL";
    case HELM_ENOMEM: return "HELM_ENOMEM";
    case HELM_ECUDA: return "HELM_ECUDA";
    case HELM_ENONFINITE: return "HELM_ENONFINITE";
    case HELM_ETIMEOUT: return "HELM_ETIMEOUT";
    case HELM_EUNSUPPORTED: return "HELM_EUNSUPPORTED";
    default: return "HELM_UNKNOWN";
    }
}

const char* helm_last_error(void) { return g_errbuf; }

uint64_t helm_launch_count(void) { return g_launches.load(); }

helm_status helm_selftest_conversions(int count, uint64_t seed, uint64_t* mismatches)
{
    if (count <= 0 || !mismatches) return HELM_EINVAL;
    unsigned long long bad = 0;
    HELM_CK(run_fp_bits_check(count, (unsigned long long)seed, &bad));
    *mismatches = bad;
    return HELM_OK;
}

helm_status helm_measure_fp64_rate(double* tflops, double* ms)
{
    if (!tflops || !ms) return HELM_EINVAL;
    HELM_CK(run_fp64_rate(tflops, ms));
    add_launches(6);
    return HELM_OK;
}

helm_status helm_plan_create(helm_plan** out, int ndim, const int* n, double h, double k, int bc,
                             int prec, void* cuda_stream)
{
    if (!out || !n) return HELM_EINVAL;
    *out = nullptr;
    if (ndim != 2 && ndim != 3) return HELM_EINVAL;
    if (bc != HELM_BC_DIRICHLET) return HELM_EUNSUPPORTED;
    if (prec != HELM_PREC_FP64 && prec != HELM_PREC_MIXED) return HELM_EINVAL;
    if (!(h > 0.0) || !std::isfinite(h) || !(k >= 0.0) || !std::isfinite(k)) return HELM_EINVAL;
    for (int a = 0; a < ndim; ++a)
        if (!is_pow2m1(n[a])) return HELM_EINVAL;
    for (int a = 1; a < ndim; ++a)
        if (n[a] != n[0]) return HELM_EUNSUPPORTED;
    if ((ndim == 2 && n[0] > 32767) || (ndim == 3 && n[0] > 2047)) return HELM_EUNSUPPORTED;
    std::unique_ptr<helm_plan> p(new helm_plan());
    p->D = ndim;
    p->n = n[0];
    p->prec = prec;
    p->h = h;
    p->k = k;
    p->alpha = k * k;
    p->damp = 0.0;
    p->sigma = 0.0;
    p->stream = (cudaStream_t)cuda_stream;
    helm_status st = p->eng.init(ndim, prec);
    if (st != HELM_OK) return st;
    p->eng.latency = true;                     // a plan's solve runs alone
    st = alloc_instance(p->inst, ndim, n[0], h, k, prec, 1024, p->stream, false);
    if (st != HELM_OK) return st;
    p->eng.slots[0] = &p->inst;
    p->eng.dirty = true;
    HELM_CK(cudaStreamSynchronize(p->stream));
    *out = p.release();
    return HELM_OK;
}

helm_status helm_plan_destroy(helm_plan* p)
{
    if (!p) return HELM_EINVAL;
    cudaStreamSynchronize(p->stream);
    p->eng.release();
    free_instance(p->inst, p->stream);
    delete p;
    return HELM_OK;
}

helm_status helm_plan_info(const helm_plan* p, double* lmin, double* kmax, double* rho, size_t* ws)
{
    if (!p) return HELM_EINVAL;
    const double l = lambda_min_of(p->D, p->n, p->h);
    // G = -(alpha + i p)(Delta_h - sigma)^{-1}: rho = |alpha + i p| / (lambda_min + sigma);
    // the iteration converges iff k^2 < lambda_min + alpha - |alpha + i p| (= lambda_min
    // when p = 0, whatever alpha)
    const double mod = std::hypot(p->alpha, p->damp);
    const double q = l + p->alpha - mod;
    if (lmin) *lmin = l;
    if (kmax) *kmax = p->damp == 0.0 ? std::sqrt(l) : (q > 0.0 ? std::sqrt(q) : 0.0);
    if (rho) *rho = mod / (l + p->sigma);
    if (ws) *ws = p->inst.ws_bytes + (2 * (size_t)p->inst.hist_cap + 1) * sizeof(double);
    return HELM_OK;
}

helm_status helm_plan_set_cavity(helm_plan* p, double alpha, double damp)
{
    if (!p) return HELM_EINVAL;
    if (!std::isfinite(alpha) || !std::isfinite(damp) || damp < 0.0) return HELM_EINVAL;
    if (alpha < p->k * p->k) return HELM_EINVAL;          // Section 2.2: alpha >= k^2
    const double k2 = p->k * p->k;
    p->alpha = alpha;
    p->damp = damp;
    p->sigma = (alpha == k2) ? 0.0 : alpha - k2;
    set_shift(p->inst.d, p->sigma);
    p->inst.d.damp = damp;
    return HELM_OK;
}

helm_status helm_plan_coarse(const helm_plan* p, int* tail_n, int* exact_n)
{
    if (!p) return HELM_EINVAL;
    const int tn = p->inst.d.lev[p->inst.d.ltail].n;
    const int xn = tail_exact_n(p->D, p->prec == HELM_PREC_FP64 ? 0 : 1);
    if (tail_n) *tail_n = tn;
    if (exact_n) *exact_n = (xn > 0 && tn >= xn) ? xn : 0;
    return HELM_OK;
}

helm_status helm_exit_time(helm_plan* p, double tol, int max_outer, void* E_out, double* emax,
                           double* kstar)
{
    if (!p || !(tol >= 0.0) || max_outer < 1) return HELM_EINVAL;
    if (E_out && check_ptr(E_out)) return HELM_EINVAL;
    // Delta_h E = -1, E = 0 on the wall: the outer iteration with k = 0 (its steps are
    // multigrid cycles refined in FP64), on a plan of the same geometry and precision
    helm_plan* q = nullptr;
    const int nn[3] = {p->n, p->n, p->n};
    helm_status st = helm_plan_create(&q, p->D, nn, p->h, 0.0, HELM_BC_DIRICHLET, p->prec, p->stream);
    if (st != HELM_OK) return st;
    q->eng.nu1 = p->eng.nu1;
    q->eng.nu2 = p->eng.nu2;
    q->eng.cycles = p->eng.cycles;
    const size_t fb = p->points() * 16, ub = p->padded() * 16;
    char* buf = nullptr;
    if (cudaMalloc((void**)&buf, fb + 2 * ub + 256) != cudaSuccess) {
        cudaGetLastError();
        helm_plan_destroy(q);
        return HELM_ENOMEM;
    }
    void* f = buf;
    void* g = buf + fb;
    void* u = buf + fb + ub;
    unsigned long long* dmax = (unsigned long long*)(buf + fb + 2 * ub);
    auto done = [&](helm_status s) { cudaFree(buf); helm_plan_destroy(q); return s; };
    if (launch_fill_c128(f, (long)p->points(), -1.0, 0.0, p->stream) != cudaSuccess ||
        cudaMemsetAsync(g, 0, 2 * ub + 256, p->stream) != cudaSuccess)
        return done(HELM_ECUDA);
    int iters = 0;
    st = helm_solve(q, f, g, u, tol, max_outer, &iters, nullptr);
    if (st < 0) return done(st);
    unsigned long long bits = 0;
    if (launch_max_re(p->D, p->n, u, dmax, p->stream) != cudaSuccess ||
        cudaMemcpyAsync(&bits, dmax, sizeof bits, cudaMemcpyDeviceToHost, p->stream) != cudaSuccess)
        return done(HELM_ECUDA);
    if (E_out && cudaMemcpyAsync(E_out, u, ub, cudaMemcpyDeviceToDevice, p->stream) != cudaSuccess)
        return done(HELM_ECUDA);
    if (cudaStreamSynchronize(p->stream) != cudaSuccess) return done(HELM_ECUDA);
    g_launches += 2;
    double m;
    memcpy(&m, &bits, sizeof m);
    if (emax) *emax = m;
    if (kstar) {
        const double r = (m > 0.0) ? 1.0 / m - p->damp : -1.0;
        *kstar = r > 0.0 ? std::sqrt(r) : 0.0;
    }
    return done(st);
}

helm_status helm_plan_set_cycle(helm_plan* p, int nu1, int nu2, int cycles)
{
    if (!p) return HELM_EINVAL;
    if (nu1 < 0 || nu1 > 8 || nu2 < 0 || nu2 > 8 || nu1 + nu2 < 1 || cycles < 1 || cycles > 16)
        return HELM_EINVAL;
    p->eng.nu1 = nu1;
    p->eng.nu2 = nu2;
    p->eng.cycles = cycles;
    p->eng.dirty = true;
    return HELM_OK;
}

helm_status helm_solve_ex(helm_plan* p, const void* f, const void* g, void* u, double tol,
                          int max_outer, int* iters, double* res_hist, double* einf_hist)
{
    if (!p) return HELM_EINVAL;
    if (max_outer < 0 || !(tol >= 0.0)) return HELM_EINVAL;
    if (check_ptr(f) || check_ptr(g) || check_ptr(u)) return HELM_EINVAL;
    const size_t fb = p->points() * 16, ub = p->padded() * 16;
    if (overlap(f, fb, u, ub) || overlap(g, ub, u, ub)) return HELM_EINVAL;
    Instance& in = p->inst;
    if (max_outer > in.hist_cap) {
        HELM_CK(cudaStreamSynchronize(p->stream));
        if (in.hist_sep && in.hist) cudaFree(in.hist);   // else it lives in the workspace allocation
        in.hist = nullptr;
        in.hist_sep = false;
        const size_t hb = (2 * (size_t)max_outer + 1) * sizeof(double);
        if (cudaMalloc((void**)&in.hist, hb) != cudaSuccess) { cudaGetLastError(); return HELM_ENOMEM; }
        in.hist_sep = true;
        in.hist_cap = max_outer;
        in.d.hist = in.hist;
        in.d.einf = in.hist + max_outer + 1;
    }
    in.d.u[0] = (double2*)u;
    in.d.f = (const double2*)f;
    in.d.g = (const double2*)g;
    in.d.tol = tol;
    in.d.max_outer = max_outer;
    in.d.k2 = p->k * p->k;
    in.d.cdiag = in.d.k2 - 2.0 * p->D * in.d.ih2;
    set_shift(in.d, p->sigma);
    in.d.damp = p->damp;
    helm_status st = p->eng.prepare();
    if (st != HELM_OK) return st;
    st = p->eng.start_instance(0, p->stream);
    if (st != HELM_OK) return st;
    int steps = 0;
    st = p->eng.run(p->stream, 0, &steps);
    if (st != HELM_OK) return st;
    const InstState s = p->eng.h_state[0];
    if (s.it & 1) HELM_CK(cudaMemcpyAsync(u, in.d.u[1], ub, cudaMemcpyDeviceToDevice, p->stream));
    if (res_hist) HELM_CK(cudaMemcpyAsync(res_hist, in.d.hist, (s.it + 1) * sizeof(double),
                                          cudaMemcpyDeviceToHost, p->stream));
    if (einf_hist && s.it > 0)
        HELM_CK(cudaMemcpyAsync(einf_hist, in.d.einf, s.it * sizeof(double), cudaMemcpyDeviceToHost,
                                p->stream));
    HELM_CK(cudaStreamSynchronize(p->stream));
    // leave the slot idle so standalone V-cycles see a known state
    InstState idle;
    memset(&idle, 0, sizeof idle);
    idle.status = HELM_ST_IDLE;
    HELM_CK(cudaMemcpy(p->eng.d_state, &idle, sizeof idle, cudaMemcpyHostToDevice));
    if (iters) *iters = s.it;
    return (helm_status)s.status;
}

helm_status helm_solve(helm_plan* p, const void* f, const void* g, void* u, double tol,
                       int max_outer, int* iters, double* res_hist)
{
    return helm_solve_ex(p, f, g, u, tol, max_outer, iters, res_hist, nullptr);
}

helm_status helm_plan_autotune(helm_plan* p, const void* f, const void* g, void* u, double tol,
                               int max_outer, int* nu1_out, int* nu2_out, int* cycles_out,
                               double* best_ms)
{
    if (!p) return HELM_EINVAL;
    if (check_ptr(f) || check_ptr(g) || check_ptr(u)) return HELM_EINVAL;
    static const int cand[][3] = {{1, 0, 1}, {0, 1, 1}, {0, 2, 1}, {0, 3, 1}, {1, 1, 1}, {2, 1, 1},
                                  {1, 2, 1}, {2, 2, 1}, {3, 3, 1}, {1, 1, 2}};
    const size_t ub = p->padded() * 16;
    void* saved = nullptr;
    HELM_CK(cudaMallocAsync(&saved, ub, p->stream));
    HELM_CK(cudaMemcpyAsync(saved, u, ub, cudaMemcpyDeviceToDevice, p->stream));
    cudaEvent_t e0, e1;
    HELM_CK(cudaEventCreate(&e0));
    HELM_CK(cudaEventCreate(&e1));
    const int s1 = p->eng.nu1, s2 = p->eng.nu2, sc = p->eng.cycles, st0 = p->eng.tiles, cm0 = p->eng.coarse;
    // best of two timed solves after a first one that builds the graph; HELM_CONVERGED and
    // the time, or the first solve's outcome
    auto time_solve = [&](float* ms_out) -> helm_status {
        float best = 0.f;
        for (int rep = 0; rep < 3; ++rep) {
            HELM_CK(cudaMemcpyAsync(u, saved, ub, cudaMemcpyDeviceToDevice, p->stream));
            HELM_CK(cudaEventRecord(e0, p->stream));
            const helm_status out = helm_solve(p, f, g, u, tol, max_outer, nullptr, nullptr);
            HELM_CK(cudaEventRecord(e1, p->stream));
            HELM_CK(cudaEventSynchronize(e1));
            if (out != HELM_CONVERGED) return out;
            float ms = 0.f;
            HELM_CK(cudaEventElapsedTime(&ms, e0, e1));
            if (rep > 0 && (best == 0.f || ms < best)) best = ms;
        }
        *ms_out = best;
        return HELM_CONVERGED;
    };
    int bi = -1, bt = st0, bc = cm0;
    float bms = 0.f;
    helm_status st = HELM_OK;
    for (int c = 0; c < (int)(sizeof cand / sizeof cand[0]); ++c) {
        st = helm_plan_set_cycle(p, cand[c][0], cand[c][1], cand[c][2]);
        if (st != HELM_OK) break;
        float ms = 0.f;
        const helm_status out = time_solve(&ms);
        if (out < 0) { st = out; break; }
        if (out == HELM_CONVERGED && (bi < 0 || ms < bms)) {
            bi = c;
            bms = ms;
        }
    }
    // 2D: the tile-shape policies of the fused level kernels, with the chosen schedule
    if (st == HELM_OK && bi >= 0 && p->D == 2) {
        helm_plan_set_cycle(p, cand[bi][0], cand[bi][1], cand[bi][2]);
        for (int pol = HELM_TILES_AUTO; pol <= HELM_TILES_SMALL; ++pol) {
            if (pol == st0) continue;
            p->eng.tiles = pol;
            p->eng.dirty = true;
            float ms = 0.f;
            const helm_status out = time_solve(&ms);
            if (out < 0) { st = out; break; }
            if (out == HELM_CONVERGED && ms < bms) {
                bt = pol;
                bms = ms;
            }
        }
    }
    // 2D complex64: the one-CTA coarse tail against the cluster tail (where it applies)
    if (st == HELM_OK && bi >= 0 && p->D == 2 && p->prec != HELM_PREC_FP64) {
        p->eng.tiles = bt;
        for (int cm = HELM_COARSE_AUTO; cm <= HELM_COARSE_CLUSTER; ++cm) {
            if (cm == cm0) continue;
            p->eng.coarse = cm;
            p->eng.dirty = true;
            float ms = 0.f;
            const helm_status out = time_solve(&ms);
            if (out < 0) { st = out; break; }
            if (out == HELM_CONVERGED && ms < bms) {
                bc = cm;
                bms = ms;
            }
        }
    }
    HELM_CK(cudaMemcpyAsync(u, saved, ub, cudaMemcpyDeviceToDevice, p->stream));
    HELM_CK(cudaFreeAsync(saved, p->stream));
    HELM_CK(cudaStreamSynchronize(p->stream));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != HELM_OK || bi < 0) {                         // error, or nothing converged: keep the old schedule
        helm_plan_set_cycle(p, s1, s2, sc);
        p->eng.tiles = st0;
        p->eng.coarse = cm0;
        p->eng.dirty = true;
        return st != HELM_OK ? st : HELM_DIVERGED;
    }
    helm_plan_set_cycle(p, cand[bi][0], cand[bi][1], cand[bi][2]);
    p->eng.tiles = bt;
    p->eng.coarse = bc;
    p->eng.dirty = true;
    if (nu1_out) *nu1_out = cand[bi][0];
    if (nu2_out) *nu2_out = cand[bi][1];
    if (cycles_out) *cycles_out = cand[bi][2];
    if (best_ms) *best_ms = bms;
    return HELM_OK;
}

helm_status helm_plan_set_tiles(helm_plan* p, int policy)
{
    if (!p || policy < HELM_TILES_AUTO || policy > HELM_TILES_SMALL) return HELM_EINVAL;
    p->eng.tiles = policy;
    p->eng.dirty = true;
    return HELM_OK;
}

helm_status helm_plan_tiles(const helm_plan* p, int* policy)
{
    if (!p || !policy) return HELM_EINVAL;
    *policy = p->eng.tiles;
    return HELM_OK;
}

helm_status helm_plan_set_coarse_mode(helm_plan* p, int mode)
{
    if (!p || mode < HELM_COARSE_AUTO || mode > HELM_COARSE_CLUSTER) return HELM_EINVAL;
    p->eng.coarse = mode;
    p->eng.dirty = true;
    return HELM_OK;
}

helm_status helm_plan_coarse_mode(const helm_plan* p, int* mode, int* cluster_used)
{
    if (!p || !mode) return HELM_EINVAL;
    *mode = p->eng.coarse;
    if (cluster_used) {
        int used = 0;
        for (const LaunchRec& L : p->eng.step) used |= (L.kind == LaunchRec::CTAIL) ? 1 : 0;
        *cluster_used = used;
    }
    return HELM_OK;
}

helm_status helm_spectral_radius(helm_plan* p, int max_iters, double tol, int cycles, double* rho,
                                 int* iters_done)
{
    if (!p || max_iters < 1 || !(tol >= 0.0) || cycles < 1 || cycles > 64) return HELM_EINVAL;
    Engine& E = p->eng;
    const int pr = p->prec == HELM_PREC_FP64 ? 0 : 1;
    // one V-cycle of the plan's schedule from the current iterate, on instance 0
    const int sc = E.cycles;
    E.cycles = 1;
    helm_status st = E.rebuild_plan();
    E.cycles = sc;
    E.dirty = true;
    E.plan_sig.clear();
    E.graph_sig.clear();
    if (st != HELM_OK) return st;
    double* buf = nullptr;
    const int nb = power_iteration_blocks();
    if (cudaMalloc((void**)&buf, (nb + 1) * sizeof(double)) != cudaSuccess) { cudaGetLastError(); return HELM_ENOMEM; }
    InstState act;
    memset(&act, 0, sizeof act);
    act.status = HELM_ST_ACTIVE;
    const double npts = (double)p->points();
    double mu = 0.0, prev = -1.0;
    int it = 0;
    auto fail = [&](helm_status s) { cudaFree(buf); return s; };
    if (cudaMemcpyAsync(E.d_desc, &p->inst.d, sizeof(InstDesc), cudaMemcpyHostToDevice, p->stream) != cudaSuccess ||
        cudaMemcpyAsync(E.d_state, &act, sizeof act, cudaMemcpyHostToDevice, p->stream) != cudaSuccess ||
        launch_lev_fill(p->D, pr, E.d_desc, 1, 1.0 / std::sqrt(npts), p->stream) != cudaSuccess)
        return fail(HELM_ECUDA);
    while (it < max_iters) {
        ++it;
        // w = M^{-1} v by `cycles` cycles from zero (M = Delta_h - sigma, zero walls)
        if (launch_lev_fill(p->D, pr, E.d_desc, 0, 0.0, p->stream) != cudaSuccess) return fail(HELM_ECUDA);
        for (int c = 0; c < cycles; ++c) {
            st = E.enqueue(E.vcyc_plain, p->stream, false);
            if (st != HELM_OK) return fail(st);
        }
        double s2 = 0.0;
        if (launch_lev_sumsq(p->D, pr, E.d_desc, buf, buf + nb, p->stream) != cudaSuccess ||
            cudaMemcpyAsync(&s2, buf + nb, sizeof s2, cudaMemcpyDeviceToHost, p->stream) != cudaSuccess ||
            cudaStreamSynchronize(p->stream) != cudaSuccess)
            return fail(HELM_ECUDA);
        g_launches += (uint64_t)cycles * E.vcyc_plain.size() + 3;
        mu = std::sqrt(s2);                     // ||M^{-1} v|| with ||v|| = 1
        if (!(mu > 0.0) || !std::isfinite(mu)) return fail(HELM_ENONFINITE);
        if (launch_lev_scale(p->D, pr, E.d_desc, 1.0 / mu, p->stream) != cudaSuccess) return fail(HELM_ECUDA);
        if (prev > 0.0 && std::fabs(mu - prev) <= tol * mu) break;
        prev = mu;
    }
    InstState idle;
    memset(&idle, 0, sizeof idle);
    idle.status = HELM_ST_IDLE;
    cudaMemcpyAsync(E.d_state, &idle, sizeof idle, cudaMemcpyHostToDevice, p->stream);
    cudaStreamSynchronize(p->stream);
    cudaFree(buf);
    // G = -(alpha + i p) M^{-1}: |eigenvalue| = |alpha + i p| / (lambda_m + sigma)
    if (rho) *rho = std::hypot(p->alpha, p->damp) * mu;
    if (iters_done) *iters_done = it;
    return (prev > 0.0 && std::fabs(mu - prev) <= tol * mu) ? HELM_OK : HELM_MAXITER;
}

helm_status poisson_vcycle(helm_plan* p, const void* rhs, void* e, int nu1, int nu2)
{
    if (!p) return HELM_EINVAL;
    if (nu1 < 0 || nu1 > 8 || nu2 < 0 || nu2 > 8 || nu1 + nu2 < 1) return HELM_EINVAL;
    if (check_ptr(rhs) || check_ptr(e)) return HELM_EINVAL;
    const size_t b = p->points() * (size_t)elem_bytes(p->prec);
    if (overlap(rhs, b, e, b)) return HELM_EINVAL;
    Engine& E = p->eng;
    const int s1 = E.nu1, s2 = E.nu2, sc = E.cycles;
    E.nu1 = nu1;
    E.nu2 = nu2;
    E.cycles = 1;
    helm_status st = E.rebuild_plan();
    E.nu1 = s1;
    E.nu2 = s2;
    E.cycles = sc;
    E.dirty = true;
    E.plan_sig.clear();
    E.graph_sig.clear();
    if (st != HELM_OK) return st;
    InstState act;
    memset(&act, 0, sizeof act);
    act.status = HELM_ST_ACTIVE;
    HELM_CK(cudaMemcpyAsync(E.d_desc, &p->inst.d, sizeof(InstDesc), cudaMemcpyHostToDevice, p->stream));
    HELM_CK(cudaMemcpyAsync(E.d_state, &act, sizeof act, cudaMemcpyHostToDevice, p->stream));
    HELM_CK(launch_pack(p->D, p->prec == HELM_PREC_FP64 ? 0 : 1, E.d_desc, 0, p->n, rhs, 1, p->stream));
    HELM_CK(launch_pack(p->D, p->prec == HELM_PREC_FP64 ? 0 : 1, E.d_desc, 0, p->n, e, 0, p->stream));
    E.nu1 = nu1;
    E.nu2 = nu2;
    st = E.enqueue(E.vcyc_plain, p->stream, false);
    E.nu1 = s1;
    E.nu2 = s2;
    if (st != HELM_OK) return st;
    HELM_CK(launch_unpack(p->D, p->prec == HELM_PREC_FP64 ? 0 : 1, E.d_desc, 0, p->n, e, p->stream));
    InstState idle;
    memset(&idle, 0, sizeof idle);
    idle.status = HELM_ST_IDLE;
    HELM_CK(cudaMemcpyAsync(E.d_state, &idle, sizeof idle, cudaMemcpyHostToDevice, p->stream));
    HELM_CK(cudaStreamSynchronize(p->stream));
    g_launches += E.vcyc_plain.size() + 3;
    return HELM_OK;
}

// ---------------------------------------------------------------------------
// Batch / serving
// ---------------------------------------------------------------------------

helm_status helm_batch_create(helm_batch** out, size_t cap, void* stream)
{
    if (!out) return HELM_EINVAL;
    *out = nullptr;
    std::unique_ptr<helm_batch> b(new helm_batch());
    b->cap_bytes = cap;
    b->stream = (cudaStream_t)stream;
    HELM_CK(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming));
    // keep freed instance memory in the pool for the next admissions
    int dev = 0;
    HELM_CK(cudaGetDevice(&dev));
    cudaMemPool_t pool;
    HELM_CK(cudaDeviceGetDefaultMemPool(&pool, dev));
    uint64_t thr = UINT64_MAX;
    HELM_CK(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr));
    *out = b.release();
    return HELM_OK;
}

helm_status helm_batch_destroy(helm_batch* b)
{
    if (!b) return HELM_EINVAL;
    cudaStreamSynchronize(b->stream);
    for (auto& kv : b->recs)
        if (kv.second.inst) {
            free_instance(*kv.second.inst, b->stream);
            delete kv.second.inst;
        }
    cudaStreamSynchronize(b->stream);
    b->engines.clear();
    for (cudaStream_t s : b->rank_streams) cudaStreamDestroy(s);
    for (cudaEvent_t e : b->rank_join) cudaEventDestroy(e);
    if (b->up_stream) cudaStreamDestroy(b->up_stream);
    if (b->up_fork) cudaEventDestroy(b->up_fork);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->h_hist) cudaFreeHost(b->h_hist);
    if (b->h_init) cudaFreeHost(b->h_init);
    if (b->d_init) cudaFree(b->d_init);
    delete b;
    return HELM_OK;
}

static helm_status set_host_result_rec(helm_batch::Rec& r, void* host_u);

// Engines are keyed by kernel class, grid size and lane: the solves of one size share
// their engines (so every launch of an engine covers one size: the fused finest-level
// kernel, paired descents and cluster tails apply, and no phase of the level-aligned plan
// is empty for some solves), and each size's solves are spread over `lanes` engines.
constexpr int KEY_SIZES = 16;                   // log2(n + 1) <= 15
inline int engine_key(int cls, int sizeg, int lane) { return (cls * KEY_SIZES + sizeg) * HELM_MAX_LANES + lane; }
inline int engine_class(int key) { return key / (KEY_SIZES * HELM_MAX_LANES); }
inline int size_group(int n)
{
    int g = 0;
    while (g < KEY_SIZES - 1 && (2 << g) - 1 < n) ++g;
    return g + 1 < KEY_SIZES ? g + 1 : KEY_SIZES - 1;
}

// host: f, g, u are host pointers (helm_batch_submit_host): the solve's own device copies
// are part of its allocation, f and g uploaded on the batch's upload stream, u zeroed, and
// the result copied to u when the solve ends
static helm_status submit_impl(helm_batch* b, int D, int n, double h, double k, int prec,
                               const void* f, const void* g, void* u, double tol, int max_outer,
                               uint64_t* ticket, double sigma = 0.0, double damp = 0.0, bool host = false)
{
    if (!b || !ticket) return HELM_EINVAL;
    if (D != 2 && D != 3) return HELM_EINVAL;
    if (!is_pow2m1(n) || (D == 2 && n > 32767) || (D == 3 && n > 2047)) return HELM_EINVAL;
    if (!(h > 0.0) || !std::isfinite(h) || !(k >= 0.0) || !std::isfinite(k)) return HELM_EINVAL;
    if (prec != HELM_PREC_FP64 && prec != HELM_PREC_MIXED) return HELM_EINVAL;
    if (max_outer < 0 || !(tol >= 0.0)) return HELM_EINVAL;
    const size_t S = (size_t)n + 2;
    const size_t fb = (D == 3 ? (size_t)n * n * n : (size_t)n * n) * 16;
    const size_t ub = (D == 3 ? S * S * S : S * S) * 16;
    if (host) {
        if (!f || !g || !u) return HELM_EINVAL;
        cudaPointerAttributes a;
        for (const void* q : {f, g, (const void*)u}) {
            if (cudaPointerGetAttributes(&a, q) != cudaSuccess) {
                cudaGetLastError();
                return HELM_EINVAL;
            }
            if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return HELM_EINVAL;
        }
    } else if (check_ptr(f) || check_ptr(g) || check_ptr(u)) {
        return HELM_EINVAL;
    }
    if (overlap(f, fb, u, ub) || overlap(g, ub, u, ub)) return HELM_EINVAL;
    const size_t io_bytes = host ? align256(fb) + 2 * align256(ub) : 0;
    InstDesc probe{};
    const size_t need = layout(probe, D, n, h, k, prec, nullptr) +
                        (2 * (size_t)max_outer + 1) * sizeof(double) + io_bytes;
    if (b->cap_bytes && b->used + need > b->cap_bytes) return HELM_ENOMEM;
    // the lane of this class and size with the least predicted work in it (solves submitted
    // longest first are then spread as longest-job-first: the longest alone, the rest
    // balanced)
    const int sg = size_group(n);
    int key = engine_key(2 * D + prec, sg, 0);
    {
        double best = 0.0;
        bool first = true;
        for (int lane = 0; lane < b->lanes; ++lane) {
            const int k2 = engine_key(2 * D + prec, sg, lane);
            auto e = b->engines.find(k2);
            const double w = (e == b->engines.end()) ? 0.0 : e->second->total_work();
            if (first || w < best) { best = w; key = k2; first = false; }
        }
    }
    Engine* E = nullptr;
    auto it = b->engines.find(key);
    if (it == b->engines.end()) {
        std::unique_ptr<Engine> ne(new Engine());
        helm_status st = ne->init(D, prec);
        if (st != HELM_OK) return st;
        const int* cs = b->cls_sched[2 * D + prec];
        ne->nu1 = cs[2] ? cs[0] : b->nu1;
        ne->nu2 = cs[2] ? cs[1] : b->nu2;
        ne->cycles = cs[2] ? cs[2] : b->cycles;
        ne->tiles = b->tiles;
        ne->coarse = b->coarse;
        E = ne.get();
        b->engines[key] = std::move(ne);
    } else {
        E = it->second.get();
    }
    int slot = -1;
    for (int i = 0; i < E->cap; ++i)
        if (!E->slots[i]) { slot = i; break; }
    if (slot < 0) {
        slot = E->cap;
        helm_status st = E->grow(E->cap + 1);
        if (st != HELM_OK) return st;
    }
    Instance* in = new Instance();
    WsInit wi{};
    helm_status st = alloc_instance(*in, D, n, h, k, prec, max_outer, b->stream, true, io_bytes, &wi);
    if (st != HELM_OK) { free_instance(*in, b->stream); delete in; return st; }
    b->init_pending.push_back(wi);
    void* ud = u;
    const void* fd = f;
    const void* gd = g;
    if (host) {
        // the device copies: the upload stream waits for the allocation (stream-ordered on
        // the batch stream), then copies f and g and zeroes u (the paper's start; the ring
        // is set from g when the solve starts); the solve's first step waits for it
        fd = in->io;
        gd = in->io + align256(fb);
        ud = in->io + align256(fb) + align256(ub);
        if (!b->up_stream) {
            HELM_CK(cudaStreamCreateWithFlags(&b->up_stream, cudaStreamNonBlocking));
            HELM_CK(cudaEventCreateWithFlags(&b->up_fork, cudaEventDisableTiming));
        }
        HELM_CK(cudaEventCreateWithFlags(&in->ready, cudaEventDisableTiming));
        HELM_CK(cudaEventRecord(b->up_fork, b->stream));
        HELM_CK(cudaStreamWaitEvent(b->up_stream, b->up_fork, 0));
        HELM_CK(cudaMemcpyAsync((void*)fd, f, fb, cudaMemcpyHostToDevice, b->up_stream));
        HELM_CK(cudaMemcpyAsync((void*)gd, g, ub, cudaMemcpyHostToDevice, b->up_stream));
        HELM_CK(cudaMemsetAsync(ud, 0, ub, b->up_stream));
        HELM_CK(cudaEventRecord(in->ready, b->up_stream));
    }
    in->d.u[0] = (double2*)ud;
    in->d.f = (const double2*)fd;
    in->d.g = (const double2*)gd;
    in->d.tol = tol;
    in->d.max_outer = max_outer;
    set_shift(in->d, sigma);
    in->d.damp = damp;
    E->slots[slot] = in;
    E->dirty = true;
    E->pending.push_back(slot);                 // started by the next step, on its lane
    helm_batch::Rec r;
    r.key = key;
    r.slot = slot;
    r.inst = in;
    r.u = ud;
    r.ubytes = ub;
    if (host) {
        st = set_host_result_rec(r, u);
        if (st != HELM_OK) return st;
    }
    const uint64_t t = b->next++;
    b->recs[t] = r;
    b->used += need;
    *ticket = t;
    return HELM_OK;
}

helm_status helm_batch_submit(helm_batch* b, const helm_plan* p, const void* f, const void* g,
                              void* u, double tol, int max_outer, uint64_t* ticket)
{
    if (!p) return HELM_EINVAL;
    return submit_impl(b, p->D, p->n, p->h, p->k, p->prec, f, g, u, tol, max_outer, ticket,
                       p->sigma, p->damp);
}

helm_status helm_batch_submit_geom(helm_batch* b, int ndim, int n, double h, double k, int prec,
                                   const void* f, const void* g, void* u, double tol,
                                   int max_outer, uint64_t* ticket)
{
    return submit_impl(b, ndim, n, h, k, prec, f, g, u, tol, max_outer, ticket);
}

helm_status helm_batch_submit_many(helm_batch* b, int count, const int* ndim, const int* n, const double* h,
                                   const double* k, int prec, const void* const* f, const void* const* g,
                                   void* const* u, double tol, int max_outer, uint64_t* tickets, int* admitted)
{
    if (!b || count < 0 || !admitted || (count > 0 && (!ndim || !n || !h || !k || !f || !g || !u || !tickets)))
        return HELM_EINVAL;
    *admitted = 0;
    for (int i = 0; i < count; ++i) {
        const helm_status st = submit_impl(b, ndim[i], n[i], h[i], k[i], prec, f[i], g[i], u[i], tol, max_outer,
                                           &tickets[i]);
        if (st != HELM_OK) return st;                 // HELM_ENOMEM: the rest wait for retirements
        *admitted = i + 1;
    }
    return HELM_OK;
}

helm_status helm_batch_poll_many(helm_batch* b, int count, const uint64_t* tickets, int release, int* done,
                                 int* status, int* iters)
{
    if (!b || count < 0 || (count > 0 && (!tickets || !done))) return HELM_EINVAL;
    for (int i = 0; i < count; ++i) {
        auto it = b->recs.find(tickets[i]);
        if (it == b->recs.end()) return HELM_EINVAL;
        helm_batch::Rec& r = it->second;
        done[i] = r.done;
        if (!r.done) continue;
        if (status) status[i] = r.status;
        if (iters) iters[i] = r.iters;
        if (release) b->recs.erase(it);
    }
    return HELM_OK;
}

static helm_status retire_finished(helm_batch* b)
{
    // retire finished instances: result into the caller's u, histories to the host
    std::vector<helm_batch::Rec*> fin;
    size_t nh = 0;
    for (auto& kv : b->recs) {
        helm_batch::Rec& r = kv.second;
        if (r.done || !r.inst) continue;
        Engine* E = b->engines[r.key].get();
        const InstState s = E->h_state[r.slot];
        if (s.status == HELM_ST_ACTIVE || s.status == HELM_ST_IDLE) continue;
        fin.push_back(&r);
        nh += (size_t)s.it + 1;
    }
    if (fin.empty()) return HELM_OK;
    if (nh > b->h_hist_cap) {
        if (b->h_hist) cudaFreeHost(b->h_hist);
        b->h_hist = nullptr;
        b->h_hist_cap = 0;
        HELM_CK(cudaMallocHost(&b->h_hist, nh * sizeof(double)));
        b->h_hist_cap = nh;
    }
    size_t off = 0;
    for (helm_batch::Rec* rp : fin) {
        helm_batch::Rec& r = *rp;
        const InstState s = b->engines[r.key]->h_state[r.slot];
        if ((s.it & 1) && !r.host_sent)
            HELM_CK(cudaMemcpyAsync(r.u, r.inst->d.u[1], r.ubytes, cudaMemcpyDeviceToDevice, b->stream));
        if (r.host_u && !r.host_sent)
            HELM_CK(cudaMemcpyAsync(r.host_u, r.u, r.ubytes, cudaMemcpyDeviceToHost, b->stream));
        HELM_CK(cudaMemcpyAsync(b->h_hist + off, r.inst->d.hist, (s.it + 1) * sizeof(double),
                                cudaMemcpyDeviceToHost, b->stream));
        off += (size_t)s.it + 1;
        r.status = s.status;
        r.iters = s.it;
    }
    HELM_CK(cudaStreamSynchronize(b->stream));
    off = 0;
    for (helm_batch::Rec* rp : fin) {
        helm_batch::Rec& r = *rp;
        r.hist.assign(b->h_hist + off, b->h_hist + off + r.iters + 1);
        off += (size_t)r.iters + 1;
    }
    for (helm_batch::Rec* rp : fin) {
        helm_batch::Rec& r = *rp;
        Engine* E = b->engines[r.key].get();
        E->h_state[r.slot].status = HELM_ST_IDLE;
        HELM_CK(cudaMemcpyAsync(E->d_state + r.slot, &E->h_state[r.slot], sizeof(InstState),
                                cudaMemcpyHostToDevice, b->stream));
        InstDesc probe{};
        b->used -= layout(probe, r.inst->d.D, r.inst->d.n, r.inst->d.h, 0.0, r.inst->prec, nullptr) +
                   (2 * (size_t)r.inst->hist_cap + 1) * sizeof(double) + r.inst->io_bytes;
        free_instance(*r.inst, b->stream);
        delete r.inst;
        r.inst = nullptr;
        r.done = 1;
        E->slots[r.slot] = nullptr;
        E->dirty = true;
    }
    HELM_CK(cudaStreamSynchronize(b->stream));
    return HELM_OK;
}

helm_status helm_batch_set_lanes(helm_batch* b, int lanes)
{
    if (!b || lanes < 1 || lanes > HELM_MAX_LANES) return HELM_EINVAL;
    b->lanes = lanes;
    return HELM_OK;
}

helm_status helm_batch_set_tiles(helm_batch* b, int policy)
{
    if (!b || policy < HELM_TILES_AUTO || policy > HELM_TILES_SMALL) return HELM_EINVAL;
    b->tiles = policy;
    for (auto& kv : b->engines) {
        kv.second->tiles = policy;
        kv.second->dirty = true;
        kv.second->plan_sig.clear();
    }
    return HELM_OK;
}

helm_status helm_batch_set_coarse_mode(helm_batch* b, int mode)
{
    if (!b || mode < HELM_COARSE_AUTO || mode > HELM_COARSE_CLUSTER) return HELM_EINVAL;
    b->coarse = mode;
    for (auto& kv : b->engines) {
        kv.second->coarse = mode;
        kv.second->dirty = true;
        kv.second->plan_sig.clear();
    }
    return HELM_OK;
}

helm_status helm_batch_set_cycle_class(helm_batch* b, int ndim, int prec, int nu1, int nu2, int cycles)
{
    if (!b || (ndim != 2 && ndim != 3) || (prec != HELM_PREC_FP64 && prec != HELM_PREC_MIXED)) return HELM_EINVAL;
    if (nu1 < 0 || nu1 > 8 || nu2 < 0 || nu2 > 8 || nu1 + nu2 < 1 || cycles < 1 || cycles > 16)
        return HELM_EINVAL;
    const int c = 2 * ndim + prec;
    b->cls_sched[c][0] = nu1;
    b->cls_sched[c][1] = nu2;
    b->cls_sched[c][2] = cycles;
    for (auto& kv : b->engines) {
        if (engine_class(kv.first) != c) continue;
        kv.second->nu1 = nu1;
        kv.second->nu2 = nu2;
        kv.second->cycles = cycles;
        kv.second->dirty = true;
        kv.second->plan_sig.clear();
    }
    return HELM_OK;
}

helm_status helm_batch_set_cycle(helm_batch* b, int nu1, int nu2, int cycles)
{
    if (!b) return HELM_EINVAL;
    if (nu1 < 0 || nu1 > 8 || nu2 < 0 || nu2 > 8 || nu1 + nu2 < 1 || cycles < 1 || cycles > 16)
        return HELM_EINVAL;
    b->nu1 = nu1;
    b->nu2 = nu2;
    b->cycles = cycles;
    memset(b->cls_sched, 0, sizeof b->cls_sched);       // one schedule for every class again
    for (auto& kv : b->engines) {
        kv.second->nu1 = nu1;
        kv.second->nu2 = nu2;
        kv.second->cycles = cycles;
        kv.second->dirty = true;
        kv.second->plan_sig.clear();
    }
    return HELM_OK;
}

// the caller's u := the final iterate when it lives in the library's buffer (odd step count)
__global__ void k_final_u(const InstState* __restrict__ st, double2* __restrict__ u0,
                          const double2* __restrict__ u1, long count)
{
    if (!(st->it & 1)) return;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < count; i += (long)gridDim.x * blockDim.x)
        u0[i] = u1[i];
}

// the stream (and its join event) of launch rank r: priority decreasing with r down to
// the device's lowest (created on first use)
static helm_status rank_stream(helm_batch* b, int r, cudaStream_t* s, cudaEvent_t* e)
{
    while ((int)b->rank_streams.size() <= r) {
        const int q = (int)b->rank_streams.size();
        int least = 0, greatest = 0;
        HELM_CK(cudaDeviceGetStreamPriorityRange(&least, &greatest));
        // numerically smaller is higher priority
        const int prio = g_lane_priority ? std::min(least, greatest + q) : least;
        cudaStream_t ns;
        HELM_CK(cudaStreamCreateWithPriority(&ns, cudaStreamNonBlocking, prio));
        b->rank_streams.push_back(ns);
        cudaEvent_t ev;
        HELM_CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        b->rank_join.push_back(ev);
    }
    *s = b->rank_streams[r];
    *e = b->rank_join[r];
    return HELM_OK;
}

// The workspace set-up of the solves submitted since the batch last ran, in one launch on
// the batch stream (the lanes fork from it after this).  The staging buffer is reused only
// after the previous step's closing synchronisation.
static helm_status flush_init(helm_batch* b)
{
    const size_t n = b->init_pending.size();
    if (n == 0) return HELM_OK;
    if (n > b->init_cap) {
        if (b->h_init) cudaFreeHost(b->h_init);
        if (b->d_init) cudaFree(b->d_init);
        b->h_init = nullptr;
        b->d_init = nullptr;
        b->init_cap = 0;
        HELM_CK(cudaMallocHost(&b->h_init, n * sizeof(WsInit)));
        HELM_CK(cudaMalloc(&b->d_init, n * sizeof(WsInit)));
        b->init_cap = n;
    }
    memcpy(b->h_init, b->init_pending.data(), n * sizeof(WsInit));
    HELM_CK(cudaMemcpyAsync(b->d_init, b->h_init, n * sizeof(WsInit), cudaMemcpyHostToDevice, b->stream));
    HELM_CK(launch_init_workspaces(b->d_init, (int)n, b->stream));
    g_launches += (n + 65534) / 65535;
    b->init_pending.clear();
    return HELM_OK;
}

// The engines with work, longest predicted job first (the launch order of a step and the
// priority order of its streams).  The first is the step's critical path: holding a single
// solve, it runs in latency mode (Engine::latency); the others do not.
static std::vector<int> rank_engines(helm_batch* b)
{
    std::vector<std::pair<double, int>> order;
    for (auto& kv : b->engines)
        if (kv.second->active_count() > 0) order.push_back({kv.second->longest_job(), kv.first});
    std::stable_sort(order.begin(), order.end(),
                     [](const std::pair<double, int>& x, const std::pair<double, int>& y) { return x.first > y.first; });
    std::vector<int> keys;
    for (size_t r = 0; r < order.size(); ++r) {
        Engine* E = b->engines[order[r].second].get();
        E->latency = r == 0 && E->active_count() == 1;
        keys.push_back(order[r].second);
    }
    return keys;
}

helm_status helm_batch_step(helm_batch* b, int max_steps)
{
    if (!b || max_steps < 0) return HELM_EINVAL;
    {
        const helm_status st = flush_init(b);
        if (st != HELM_OK) return st;
    }
    // launch every engine with work on its own stream, forked from the batch stream; the
    // engine with the longest predicted job on the highest-priority stream
    HELM_CK(cudaEventRecord(b->fork, b->stream));
    const std::vector<int> order = rank_engines(b);
    std::vector<int> launched;
    for (size_t r = 0; r < order.size(); ++r) {
        const int key = order[r];
        Engine* E = b->engines[key].get();
        cudaStream_t es;
        cudaEvent_t ej;
        {
            helm_status st = rank_stream(b, (int)r, &es, &ej);
            if (st != HELM_OK) return st;
            HELM_CK(cudaStreamWaitEvent(es, b->fork, 0));
            st = E->start_pending(es);
            if (st != HELM_OK) return st;
        }
        helm_status st = E->prepare_plan();
        if (st != HELM_OK) return st;
        // A bounded chunk after a membership change runs as direct launches (finished
        // instances' kernels exit at once); the graph is (re)captured only for runs to
        // completion, so a serving loop that admits between chunks never waits on a capture.
        const bool direct = max_steps > 0 && max_steps <= 64 && !E->graph_current();
        if (!direct) {
            st = E->prepare();
            if (st != HELM_OK) return st;
        }
        E->h_ctrl[0] = 0;
        E->h_ctrl[1] = max_steps > 0 ? max_steps : INT_MAX;
        E->h_ctrl[2] = 1;
        E->h_ctrl[3] = 0;
        HELM_CK(cudaMemcpyAsync(E->d_ctrl, E->h_ctrl, 4 * sizeof(int), cudaMemcpyHostToDevice, es));
        if (direct) {
            for (int k = 0; k < max_steps; ++k) {
                st = E->enqueue(E->step, es, false);
                if (st != HELM_OK) return st;
            }
        } else {
            HELM_CK(cudaGraphLaunch(E->exec, es));
        }
        // a run to completion ends every solve of the lane: their host copies go out on the
        // lane's stream now, beside the lanes still running
        if (max_steps == 0)
            for (auto& kr : b->recs) {
                helm_batch::Rec& r = kr.second;
                // (a copy into pageable memory would hold the host, and the other lanes'
                // launches, until this lane ends: those go out at retirement instead)
                if (r.key != key || r.done || !r.inst || !r.host_u || !r.host_pinned || r.host_sent) continue;
                const long count = (long)(r.ubytes / sizeof(double2));
                k_final_u<<<(int)std::min<long>((count + 255) / 256, 1216), 256, 0, es>>>(
                    E->d_state + r.slot, (double2*)r.u, r.inst->d.u[1], count);
                HELM_CK(cudaGetLastError());
                HELM_CK(cudaMemcpyAsync(r.host_u, r.u, r.ubytes, cudaMemcpyDeviceToHost, es));
                r.host_sent = true;
            }
        HELM_CK(cudaMemcpyAsync(E->h_ctrl, E->d_ctrl, 3 * sizeof(int), cudaMemcpyDeviceToHost, es));
        HELM_CK(cudaMemcpyAsync(E->h_state, E->d_state, sizeof(InstState) * E->cap,
                                cudaMemcpyDeviceToHost, es));
        HELM_CK(cudaEventRecord(ej, es));
        HELM_CK(cudaStreamWaitEvent(b->stream, ej, 0));
        launched.push_back(key);
    }
    HELM_CK(cudaStreamSynchronize(b->stream));
    for (int key : launched) {
        Engine* E = b->engines[key].get();
        g_launches += (uint64_t)E->h_ctrl[0] * E->step.size();
    }
    return retire_finished(b);
}

helm_status helm_batch_profile(helm_batch* b, int max_steps, uint64_t* launches, double* ms,
                               double* bytes, int nkinds)
{
    if (!b || max_steps < 0 || !launches || !ms || !bytes || nkinds < (int)LaunchRec::NKINDS)
        return HELM_EINVAL;
    for (int k = 0; k < nkinds; ++k) {
        launches[k] = 0;
        ms[k] = 0.0;
        bytes[k] = 0.0;
    }
    {
        const helm_status st = flush_init(b);
        if (st != HELM_OK) return st;
    }
    for (const int key : rank_engines(b)) {
        Engine* E = b->engines[key].get();
        helm_status st = E->start_pending(b->stream);
        if (st != HELM_OK) return st;
        st = E->prepare_plan();
        if (st != HELM_OK) return st;
        const size_t nl = E->step.size();
        std::vector<cudaEvent_t> ev(2 * nl);
        for (auto& x : ev) HELM_CK(cudaEventCreate(&x));
        E->h_ctrl[0] = 0;
        E->h_ctrl[1] = INT_MAX;
        E->h_ctrl[2] = 1;
        E->h_ctrl[3] = 0;
        HELM_CK(cudaMemcpyAsync(E->d_ctrl, E->h_ctrl, 4 * sizeof(int), cudaMemcpyHostToDevice, b->stream));
        HELM_CK(cudaMemcpyAsync(E->h_state, E->d_state, sizeof(InstState) * E->cap,
                                cudaMemcpyDeviceToHost, b->stream));
        HELM_CK(cudaStreamSynchronize(b->stream));
        for (int s = 0; (max_steps == 0 || s < max_steps) && s < 1000000; ++s) {
            std::vector<double> lb(nl);
            for (size_t i = 0; i < nl; ++i) lb[i] = E->launch_bytes(E->step[i], E->h_state);
            for (size_t i = 0; i < nl; ++i) {
                HELM_CK(cudaEventRecord(ev[2 * i], b->stream));
                std::vector<LaunchRec> one{E->step[i]};
                st = E->enqueue(one, b->stream, false);
                if (st != HELM_OK) return st;
                HELM_CK(cudaEventRecord(ev[2 * i + 1], b->stream));
            }
            HELM_CK(cudaMemcpyAsync(E->h_ctrl, E->d_ctrl, 3 * sizeof(int), cudaMemcpyDeviceToHost, b->stream));
            HELM_CK(cudaMemcpyAsync(E->h_state, E->d_state, sizeof(InstState) * E->cap,
                                    cudaMemcpyDeviceToHost, b->stream));
            HELM_CK(cudaStreamSynchronize(b->stream));
            for (size_t i = 0; i < nl; ++i) {
                float t = 0.f;
                HELM_CK(cudaEventElapsedTime(&t, ev[2 * i], ev[2 * i + 1]));
                int k = (int)E->step[i].kind;
                if (k == LaunchRec::UPRES && E->step[i].color) k = LaunchRec::UPRES1;
                launches[k] += 1;
                ms[k] += t;
                bytes[k] += lb[i];
            }
            g_launches += nl;
            if (!E->h_ctrl[2]) break;
        }
        for (auto& x : ev) cudaEventDestroy(x);
        HELM_CK(cudaMemcpyAsync(E->h_state, E->d_state, sizeof(InstState) * E->cap,
                                cudaMemcpyDeviceToHost, b->stream));
        HELM_CK(cudaStreamSynchronize(b->stream));
    }
    return retire_finished(b);
}

helm_status helm_batch_poll(helm_batch* b, uint64_t ticket, int* done, int* status, int* iters,
                            double* res_hist)
{
    if (!b) return HELM_EINVAL;
    auto it = b->recs.find(ticket);
    if (it == b->recs.end()) return HELM_EINVAL;
    helm_batch::Rec& r = it->second;
    if (done) *done = r.done;
    if (!r.done) return HELM_OK;
    if (status) *status = r.status;
    if (iters) *iters = r.iters;
    if (res_hist) memcpy(res_hist, r.hist.data(), r.hist.size() * sizeof(double));
    b->recs.erase(it);
    return HELM_OK;
}

static helm_status set_host_result_rec(helm_batch::Rec& r, void* host_u)
{
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, host_u) != cudaSuccess || a.type == cudaMemoryTypeDevice ||
        a.type == cudaMemoryTypeManaged) {
        cudaGetLastError();
        return HELM_EINVAL;
    }
    r.host_u = host_u;
    r.host_pinned = a.type == cudaMemoryTypeHost;
    r.host_sent = false;
    return HELM_OK;
}

helm_status helm_batch_set_host_result(helm_batch* b, uint64_t ticket, void* host_u)
{
    if (!b || !host_u) return HELM_EINVAL;
    auto it = b->recs.find(ticket);
    if (it == b->recs.end() || it->second.done) return HELM_EINVAL;
    return set_host_result_rec(it->second, host_u);
}

helm_status helm_batch_submit_host(helm_batch* b, const helm_plan* p, const void* f_host, const void* g_host,
                                   void* u_host, double tol, int max_outer, uint64_t* ticket)
{
    if (!p) return HELM_EINVAL;
    return submit_impl(b, p->D, p->n, p->h, p->k, p->prec, f_host, g_host, u_host, tol, max_outer, ticket,
                       p->sigma, p->damp, true);
}

helm_status helm_batch_info(const helm_batch* b, int* active, size_t* bytes)
{
    if (!b) return HELM_EINVAL;
    int a = 0;
    for (auto& kv : b->recs) a += !kv.second.done;
    if (active) *active = a;
    if (bytes) *bytes = b->used;
    return HELM_OK;
}

}  // extern "C"
