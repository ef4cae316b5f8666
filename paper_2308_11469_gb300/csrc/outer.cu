// Outer (FP64) part of the Poisson iteration: the Helmholtz residual, the iterate
// update, the norms and the convergence test.
//
// One outer step of Section 2.2's iteration in residual form:
//   r_N = f - (Delta_h + k^2 + i p) u_N    (FP64, from the FP64 iterate)
//   (Delta_h - sigma) e_N = r_N, e_N = 0 on the wall, sigma = alpha - k^2
//                                          (multigrid, inner precision)
//   u_{N+1} = u_N + e_N                    (FP64)
// i.e. (Delta_h - sigma) u_{N+1} = f - (alpha + i p) u_N, Eq. (2.6) summed; with exact
// solves e_N = v_N + i w_N.  alpha = k^2, p = 0 is the default.  The wall
// data g enters through the ring of u (the Dirichlet nodes of Section 2.4 that are moved
// to the right-hand side).
//
// The residual kernels (mode 1) fuse the update with the next residual: u_{N+1} =
// u_N + e_N is formed once per node (in shared memory for 2D tiles), written to the
// other buffer of the ping-pong pair, and r_{N+1} = f - (Delta_h + k^2) u_{N+1} is formed
// in FP64 and stored, rounded to the inner precision, as the next right-hand side.
// FP64 work is kept to the update and the stencil (GB300 runs FP64 at a small fraction
// of its FP32 rate): |e| and |r|^2 are formed in the inner precision (|r|^2 from the
// stored, rounded r).  Each tile leaves one partial sum of |r|^2 and one partial
// max |e|^2; the last tile of an instance to finish (atomic ticket) sums the partials in
// tile order (deterministic), forms relres and applies the status rule.
#include "launch.h"
#include "pdl.cuh"
#include "fp_bits.cuh"
#include "fixed_lap.cuh"
#include "sweep2d.cuh"

namespace helm {
namespace {

constexpr int NTH = 256;

// FP64 -> inner precision and back; for complex64 the format changes run on the
// integer pipes (fp_bits.cuh), leaving the FP64 pipe to the update and the stencil.
__device__ __forceinline__ float2 to_inner_f(double2 v) { return make_float2(d2f_bits(v.x), d2f_bits(v.y)); }
template <typename R> struct Inner;
template <> struct Inner<float> {
    static __device__ __forceinline__ float2 from(double2 v) { return to_inner_f(v); }
    static __device__ __forceinline__ double widen(float x) { return f2d_bits(x); }
};
template <> struct Inner<double> {
    static __device__ __forceinline__ double2 from(double2 v) { return v; }
    static __device__ __forceinline__ double widen(double x) { return x; }
};

// Status rule (the paper only reports "converges" / "diverges"; this project's reading):
// CONVERGED when relres <= tol; DIVERGED when relres > 1e4, or when N >= 20, relres has
// not decreased for 10 consecutive steps and has grown to at least twice its smallest
// value so far (stagnation at the rounding floor is not divergence); NONFINITE on NaN /
// Inf; MAXITER at max_outer.
// relres_N = ||r_N|| / ||b||, b the lifted right-hand side (f minus the wall values'
// contribution to the stencil): with the paper's zero start r_0 = b and relres_0 = 1; a
// starting iterate that already solves the system well starts with a small relres.
// mode 0: `second` is ||b||^2; mode 1: it is max |e|^2.
__device__ void finalize(const InstDesc& I, InstState* stp, double norm2, double second, int mode)
{
    InstState s = *stp;
    const double norm = sqrt(norm2);
    double rel;
    int N;
    if (mode == 0) {
        N = 0;
        const double nb = sqrt(second);
        s.norm0 = (nb > 0.0) ? nb : norm;      // zero data: measure against r_0 itself
        s.run = 0;
        rel = (norm == 0.0) ? 0.0 : norm / s.norm0;
        if (!isfinite(norm) || !isfinite(nb)) rel = norm + nb;
        s.rmin = rel;
    } else {
        s.it += 1;
        N = s.it;
        rel = norm / s.norm0;
        I.einf[N - 1] = sqrt(second);
    }
    I.hist[N] = rel;
    int out = HELM_ST_ACTIVE;
    if (!isfinite(rel)) out = -4;                                   // HELM_ENONFINITE
    else if (rel <= I.tol || (mode == 0 && norm == 0.0)) out = 0;   // CONVERGED
    else if (rel > 1e4) out = 2;                                    // DIVERGED
    else {
        if (mode != 0) s.run = (rel >= s.prev) ? s.run + 1 : 0;
        s.rmin = fmin(s.rmin, rel);
        if (N >= 20 && s.run >= 10 && rel >= 2.0 * s.rmin) out = 2; // DIVERGED
        else if (N >= I.max_outer) out = 1;                         // MAXITER
    }
    s.prev = rel;
    s.status = out;
    *stp = s;
}

// Block-wide sums / maxima in a fixed order (xor-shuffle in T, then the warps' values in
// order, in FP64).  `sum2`: the second channel is summed (mode 0, ||b||^2) instead of
// maximised (max |e|^2).  Mode 1 reduces its complex64-derived values in FP32, keeping the
// shuffle tree off the FP64 pipe; the result (thread 0) is FP64 either way.
// VT > 1: each real thread stands for VT threads of a map VT times the block's size (real
// thread j for the threads j + blockDim v); virtual warp w + (blockDim / 32) v reduces on
// real warp w with the same shuffle tree, and the virtual warps' values are summed in
// order, so the result is that of the larger block.
template <typename T, int VT = 1>
__device__ __forceinline__ void block_reduce_v(const T* av, const T* mv, double& ra, double& rm,
                                               double* sa, double* sm, bool sum2)
{
    const int nw = (int)(blockDim.x >> 5);
#pragma unroll
    for (int v = 0; v < VT; ++v) {
        T a = av[v], m = mv[v];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, o);
            const T mo = __shfl_xor_sync(0xffffffffu, m, o);
            m = sum2 ? m + mo : (m > mo ? m : mo);
        }
        const int w = (threadIdx.x >> 5) + nw * v;
        if ((threadIdx.x & 31) == 0) {
            sa[w] = (double)a;
            sm[w] = (double)m;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        ra = 0.0;
        rm = 0.0;
        for (int i = 0; i < nw * VT; ++i) {
            ra += sa[i];
            rm = sum2 ? rm + sm[i] : fmax(rm, sm[i]);
        }
    }
}

template <typename T>
__device__ __forceinline__ void block_reduce(T a, T m, double& ra, double& rm, double* sa, double* sm,
                                             bool sum2)
{
    block_reduce_v<T, 1>(&a, &m, ra, rm, sa, sm, sum2);
}

// End of an outer step, run by one whole CTA once every instance's status is final: is
// any instance still iterating?  Counts the step, applies the step budget of this launch
// and sets the loop condition of the graph's WHILE node.
__device__ void step_end(const InstState* st, int nscan, int* ctrl, int use_cond,
                         unsigned long long cond_handle)
{
    __shared__ int any_active;
    if (threadIdx.x == 0) any_active = 0;
    __syncthreads();
    int a = 0;
    for (int i = threadIdx.x; i < nscan; i += blockDim.x)
        a |= (__ldcg(&st[i].status) == HELM_ST_ACTIVE);
    if (a) atomicOr(&any_active, 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        int go = any_active;
        const int done = ctrl[0] + 1;
        ctrl[0] = done;
        if (done >= ctrl[1]) go = 0;          // step budget of this launch
        ctrl[2] = go;
        if (use_cond) cudaGraphSetConditional((cudaGraphConditionalHandle)cond_handle, go ? 1u : 0u);
    }
}

// Step control folded into the residual launch (ctrl == nullptr: not folded).  Every
// instance of the launch arrives once -- an iterating instance from the CTA that
// finalised its status, a finished one from the CTA of its first tile -- and the last
// arrival (launch-wide ticket ctrl[3]) ends the step.
struct StepCtl {
    int* ctrl;
    int nscan;                  // status entries to scan (descriptor slots)
    int ninst;                  // instances with tiles in this launch
    int use_cond;
    unsigned long long cond;
};

__device__ void step_arrive(const InstState* st, const StepCtl& c)
{
    __shared__ int last_arrival;
    if (threadIdx.x == 0) {
        __threadfence();                      // this instance's status before the ticket
        last_arrival = (atomicAdd(&c.ctrl[3], 1) == c.ninst - 1);
    }
    __syncthreads();
    if (!last_arrival) return;
    __threadfence();
    step_end(st, c.nscan, c.ctrl, c.use_cond, c.cond);
    if (threadIdx.x == 0) c.ctrl[3] = 0;
}

// The CTA that wrote an instance's last partial: sum the nb partials in tile order,
// apply the status rule, and (folded step control) arrive for the step.  The partials are
// read by the first NTH threads whatever the block size (threads beyond add zeros, which
// leaves sums and maxima of non-negative values unchanged), so a launch with larger CTAs
// reduces in the same order as the residual kernels.
// sa, sm: shared scratch of one double per warp of the CTA.
// VT: threads of the NTH-thread order per real thread (blockDim.x = NTH / VT; sa, sm hold
// NTH / 32 doubles).
template <int VT = 1>
__device__ void instance_last(const InstDesc& I, InstState* stp, int mode, const InstState* st_all,
                              const StepCtl& c, double* sa, double* sm)
{
    const int nb = I.nres_blocks;
    __threadfence();
    double ta[VT], tm[VT];
#pragma unroll
    for (int v = 0; v < VT; ++v) {
        ta[v] = 0.0;
        tm[v] = 0.0;
        const int t = threadIdx.x + (int)blockDim.x * v;
        if (t < NTH)
            for (int b = t; b < nb; b += NTH) {
                ta[v] += __ldcg(I.part + b);
                const double x = __ldcg(I.part + nb + b);
                tm[v] = (mode == 0) ? tm[v] + x : fmax(tm[v], x);
            }
    }
    __syncthreads();
    double fa = 0.0, fm = 0.0;
    block_reduce_v<double, VT>(ta, tm, fa, fm, sa, sm, mode == 0);
    if (threadIdx.x == 0) {
        finalize(I, stp, fa, fm, mode);
        *I.count = 0u;
    }
    if (c.ctrl) step_arrive(st_all, c);
}

// Write this tile's partials; the last tile of the instance reduces them all.
template <typename T>
__device__ void tile_done(const InstDesc& I, InstState* stp, int tile, T ta0, T tm0, int mode,
                          const InstState* st_all, const StepCtl& c)
{
    __shared__ double sa[NTH / 32], sm[NTH / 32];
    __shared__ int last;
    double a = 0.0, m = 0.0;
    block_reduce<T>(ta0, tm0, a, m, sa, sm, mode == 0);
    if (threadIdx.x == 0) {
        I.part[tile] = a;
        I.part[I.nres_blocks + tile] = m;
        __threadfence();
        const unsigned prev = atomicAdd(I.count, 1u);
        last = (prev == (unsigned)(I.nres_blocks - 1));
    }
    __syncthreads();
    if (!last) return;
    instance_last<1>(I, stp, mode, st_all, c, sa, sm);
}

// r = f - (Delta_h + k^2 + i p) u at one node: f - k^2 u - (numerator) / h^2, the
// Laplacian numerator (sum of the neighbours - 2D u) summed exactly in fixed point
// (fixed_lap.cuh) on the scale emax, u in FP64, and for DAMP the coupling - i p u.
// helm_resid2d_fx: FC, FA, FB, FD, FU are the fixed-point images of the 2D node and its
// four neighbours (a, b west / east, d, u south / north).
template <bool DAMP>
__device__ __forceinline__ double2 helm_resid_fx(double2 c, long long lx, long long ly, double2 fv, double mih2,
                                                 double mk2, double damp, int emax)
{
    double2 r;
    r.x = fma(fx_to_double(lx, emax), mih2, fma(c.x, mk2, fv.x));
    r.y = fma(fx_to_double(ly, emax), mih2, fma(c.y, mk2, fv.y));
    if constexpr (DAMP) {
        r.x = fma(c.y, damp, r.x);
        r.y = fma(c.x, -damp, r.y);
    }
    return r;
}

template <bool DAMP>
__device__ __forceinline__ double2 helm_resid2d_fx(double2 c, longlong2 FC, longlong2 FA, longlong2 FB,
                                                   longlong2 FD, longlong2 FU, double2 fv, double mih2,
                                                   double mk2, double damp, int emax)
{
    const long long lx = ((FA.x + FB.x) + (FD.x + FU.x)) - 4 * FC.x;
    const long long ly = ((FA.y + FB.y) + (FD.y + FU.y)) - 4 * FC.y;
    return helm_resid_fx<DAMP>(c, lx, ly, fv, mih2, mk2, damp, emax);
}

// scale exponent of a window from its largest biased exponent (see fixed_lap.cuh); -1:
// no fixed-point scale (a value above 2^1007, an infinity or a NaN)
__device__ __forceinline__ int fx_scale(int emax_raw)
{
    return emax_raw > FX_EMAX ? -1 : max(emax_raw, FX_EMIN);
}

__device__ __forceinline__ longlong2 fx_fix2(double2 v, int emax)
{
    return make_longlong2(fx_fix(v.x, emax), fx_fix(v.y, emax));
}

__device__ __forceinline__ int fx_exp2(double2 v) { return max(fx_exp(v.x), fx_exp(v.y)); }

// largest of the threads' exponents (one shared word per warp; the caller's barrier
// follows before any thread reads the result)
template <int NT>
__device__ __forceinline__ int block_max_exp(int ex, int* sx)
{
    ex = __reduce_max_sync(0xffffffffu, ex);
    if ((threadIdx.x & 31) == 0) sx[threadIdx.x >> 5] = ex;
    __syncthreads();
    int m = sx[0];
#pragma unroll
    for (int w = 1; w < NT / 32; ++w) m = max(m, sx[w]);
    return m;
}

// The residual window of a tile is its (TX + 2) x (TY + 2) nodes; its 1-node ring has
// 2 (TX + 2) + 2 TY nodes, numbered: top row, bottom row, left column, right column.
template <int TX, int TY>
__device__ __forceinline__ void ring_node(int t, int& lx, int& ly)
{
    if (t < TX + 2) { lx = t; ly = 0; }
    else if (t < 2 * (TX + 2)) { lx = t - (TX + 2); ly = TY + 1; }
    else if (t < 2 * (TX + 2) + TY) { lx = 0; ly = t - 2 * (TX + 2) + 1; }
    else { lx = TX + 1; ly = t - 2 * (TX + 2) - TY + 1; }
}

// |v|^2 of an inner-precision complex value, rounded the same way in every kernel
template <typename C>
__device__ __forceinline__ auto abs2(C v) -> decltype(v.x) { return fma(v.y, v.y, v.x * v.x); }

// ---------------------------------------------------------------------------
// 2D: 32 x 32 tiles, u_{N+1} staged in shared memory with a 1-node halo
// ---------------------------------------------------------------------------
constexpr int T2 = 32;        // residual tile width (x)
constexpr int T2Y = 32;       // residual tile height (y), a multiple of 8

// DAMP: the instance has p != 0 (decided once per tile, outside the point loop)
template <typename R, int MODE, bool DAMP>
__device__ __forceinline__ void residual2d_tile(const InstDesc* __restrict__ insts,
                                                InstState* __restrict__ st, const ResItem item,
                                                double2* U, const StepCtl& c)
{
    typedef typename C2<R>::T c2;
    const InstDesc& I = insts[item.inst];
    InstState* stp = st + item.inst;
    const InstState s = *stp;
    if (s.status != HELM_ST_ACTIVE) {           // uniform over the CTA
        if (c.ctrl && item.tx == 0 && item.ty == 0) step_arrive(st, c);
        return;
    }
    const int n = I.n;
    const int S = n + 2;
    const double2* __restrict__ uin = I.u[s.it & 1];
    double2* __restrict__ uout = I.u[(s.it + 1) & 1];
    const double2* __restrict__ f = I.f;
    const LevelDesc L0 = I.lev[0];
    const c2* __restrict__ e = (const c2*)L0.e;
    c2* __restrict__ rhs = (c2*)lev_rhs(L0, 0, MODE == 1 ? s.it + 1 : s.it);   // r_{N+1} / r_0
    const int P = L0.pitch;
    const int x0 = 1 + item.tx * T2, y0 = 1 + item.ty * T2Y;
    R emax2 = 0;
    // The window's values: u_{N+1} = u_N + e_N (mode 1) or the current iterate (mode 0).
    // Each thread's residual nodes stay in registers (FP64), the window's ring goes to
    // threads 0 .. RING - 1; the window's largest exponent sets the fixed-point scale of the
    // exact Laplacian numerators.
    constexpr int KY = T2Y / 8, RING = 2 * (T2 + 2) + 2 * T2Y;
    static_assert(RING <= NTH, "one ring node per thread");
    __shared__ int sx[NTH / 32];
    const int lx = (threadIdx.x & 31) + 1;
    double2 cv[KY];
    int ex = 0;
#pragma unroll
    for (int k = 0; k < KY; ++k) {
        const int ly = (threadIdx.x >> 5) + 8 * k + 1;
        const int gx = x0 + lx - 1, gy = y0 + ly - 1;
        double2 v = make_double2(0.0, 0.0);
        if (gx <= n + 1 && gy <= n + 1) v = uin[gy * S + gx];
        if (MODE == 1 && gx <= n && gy <= n) {
            const c2 ev = e[gy * P + gx];
            v.x += Inner<R>::widen(ev.x);
            v.y += Inner<R>::widen(ev.y);
            emax2 = fmax(emax2, abs2(ev));
        }
        cv[k] = v;
        ex = max(ex, fx_exp2(v));
    }
    int rlx = 0, rly = 0;
    double2 rv = make_double2(0.0, 0.0);
    if (threadIdx.x < RING) {
        ring_node<T2, T2Y>(threadIdx.x, rlx, rly);
        const int gx = x0 - 1 + rlx, gy = y0 - 1 + rly;
        if (gx <= n + 1 && gy <= n + 1) rv = uin[gy * S + gx];
        if (MODE == 1 && gx >= 1 && gx <= n && gy >= 1 && gy <= n) {
            const c2 ev = e[gy * P + gx];
            rv.x += Inner<R>::widen(ev.x);
            rv.y += Inner<R>::widen(ev.y);
        }
        ex = max(ex, fx_exp2(rv));
    }
    const int emx = fx_scale(block_max_exp<NTH>(ex, sx));    // uniform over the CTA
    longlong2* UF = reinterpret_cast<longlong2*>(U);
#pragma unroll
    for (int k = 0; k < KY; ++k) UF[((threadIdx.x >> 5) + 8 * k + 1) * (T2 + 2) + lx] = fx_fix2(cv[k], emx);
    if (threadIdx.x < RING) UF[rly * (T2 + 2) + rlx] = fx_fix2(rv, emx);
    __syncthreads();
    const double mih2 = -I.ih2, mk2 = -I.k2;
    const double damp = I.damp;
    R r2 = 0;
    double r2d = 0.0, b2 = 0.0;
#pragma unroll
    for (int k = 0; k < KY; ++k) {
        const int ly = (threadIdx.x >> 5) + 8 * k + 1;
        const int gx = x0 + lx - 1, gy = y0 + ly - 1;
        if (gx > n || gy > n) continue;
        const int o = ly * (T2 + 2) + lx;
        const double2 c = cv[k];
        if (MODE == 1) uout[gy * S + gx] = c;
        const double2 fv = f[(size_t)(gy - 1) * n + (gx - 1)];
        const longlong2 A = UF[o - 1], Bq = UF[o + 1], Dq = UF[o - (T2 + 2)], Uq = UF[o + (T2 + 2)];
        const double2 r = (emx >= 0) ? helm_resid2d_fx<DAMP>(c, UF[o], A, Bq, Dq, Uq, fv, mih2, mk2, damp, emx)
                                     : make_double2(fx_nan(), fx_nan());
        const c2 ri = Inner<R>::from(r);
        rhs[gy * P + gx] = ri;
        if (MODE == 1) {
            r2 += abs2(ri);
        } else {
            // once per solve, in FP64: ||r_0||^2 and ||b||^2, b = f - (wall neighbours) / h^2,
            // formed with the same operations as r, so that r_0 = b bit for bit from a zero
            // start (the numerator then holds the wall values alone)
            r2d += r.x * r.x + r.y * r.y;
            double bx = fv.x, by = fv.y;            // b = f away from the wall
            if ((gx == 1 || gx == n || gy == 1 || gy == n) && emx >= 0) {
                const longlong2 z = make_longlong2(0, 0);
                const longlong2 aw = (gx == 1) ? A : z, bw = (gx == n) ? Bq : z;
                const longlong2 dw = (gy == 1) ? Dq : z, uw = (gy == n) ? Uq : z;
                const double2 bb = helm_resid2d_fx<false>(make_double2(0.0, 0.0), z, aw, bw, dw, uw, fv, mih2,
                                                          mk2, 0.0, emx);
                bx = bb.x;
                by = bb.y;
            }
            b2 += bx * bx + by * by;
        }
    }
    if constexpr (MODE == 0)
        tile_done<double>(I, stp, item.ty * I.res_tx + item.tx, r2d, b2, MODE, st, c);
    else
        tile_done<R>(I, stp, item.ty * I.res_tx + item.tx, r2, emax2, MODE, st, c);
}

// Grid-stride over the tiles of every instance (one tile per CTA when the grid covers
// them all).  DAMP: some instance of the launch has p != 0 (the others add p = 0).
// 5 resident CTAs per SM (48 registers, no spills) keep more FP64 work in flight.
template <typename R, int MODE, bool DAMP>
__global__ void __launch_bounds__(NTH, 5)
k_residual2d(const InstDesc* __restrict__ insts, InstState* __restrict__ st,
             const ResItem* __restrict__ items, int nitems, StepCtl c)
{
    __shared__ double2 U[(T2 + 2) * (T2Y + 2)];
    pdl_wait();
    pdl_trigger();
    for (int t = blockIdx.x; t < nitems; t += gridDim.x) {
        residual2d_tile<R, MODE, DAMP>(insts, st, items[t], U, c);
        __syncthreads();                          // U is restaged by the next tile
    }
}

// ---------------------------------------------------------------------------
// 2D, complex64 inner solves: level 0's ascent fused with the residual launch
// ---------------------------------------------------------------------------
// An outer step ends with level 0's prolongation + correction + nu2 sweeps (k_up2d),
// whose only reader is the residual launch.  k_upres2d does both on a 32 x 32 tile: the
// sweeps run on a window one node wider than the ascent's (halo 2 nu2 + 1), so e_N is
// final on the tile plus a 1-node ring; u_{N+1} = u_N + e_N is formed there in shared
// memory, written once, and r_{N+1} follows from the staged values.  e_N never goes to
// global memory.  The tile is one of the residual kernel's 32 x 32 tiles, and its partials
// are formed with the residual kernel's per-node arithmetic, node-to-thread map and
// summation order, so iterates, residuals and the relres history are those of the
// two-launch path bit for bit.  Level 0 keeps r_N and
// r_{N+1} in separate buffers (step parity), so tiles still sweeping with r_N never see
// another tile's r_{N+1}.
// The tile is one residual tile of k_residual2d; NTU threads (128 or 256) each stand for
// 256 / NTU threads of that kernel's map, so partials are formed in its order.
constexpr int UPY = T2Y;

// The coarse window: fine nodes gx0 .. gx0 + W - 1 (gx0 = x0 - H even when H is odd) read
// coarse X = gx >> 1 .. (gx + 1) >> 1, i.e. W / 2 + 1 columns from cx0 = gx0 >> 1.
template <int NU, int UX> constexpr int upres_cw() { return (UX + 2 * (2 * NU + 1)) / 2 + 1; }
template <int NU> constexpr int upres_ch() { return (UPY + 2 * (2 * NU + 1)) / 2 + 1; }

// u_N is staged once the sweeps are done, into the space of the rhs planes and the coarse
// window (dead by then): the CTA needs the iterate planes plus the larger of the two, which
// lets 6 CTAs share an SM instead of 5.
constexpr bool UPRES_LATE_U = true;

// With level 1 fused (L1F), level 1's final iterate on the coarse window comes from its own
// ascent formed in the tile: level 2's iterate on the window W2 below it, level 1's rhs and
// prolonged iterate on the coarse window widened by 2 nu2 nodes each side (W1).
template <int NU, int UX> constexpr int upres_w1x() { return upres_cw<NU, UX>() + 4 * NU; }
template <int NU> constexpr int upres_w1y() { return upres_ch<NU>() + 4 * NU; }
template <int NU, int UX> constexpr int upres_w2x() { return upres_w1x<NU, UX>() / 2 + 2; }
template <int NU> constexpr int upres_w2y() { return upres_w1y<NU>() / 2 + 2; }

template <int NU, int UX, bool L1F = false> constexpr size_t upres_bytes()
{
    constexpr int H = 2 * NU + 1, W = UX + 2 * H, HH = UPY + 2 * H;
    constexpr size_t ub = (size_t)(UX + 2) * (UPY + 2) * sizeof(double2);
    constexpr size_t planes = (size_t)W * HH * sizeof(float2);          // E0 + E1 (or R0 + R1)
    constexpr size_t cs = L1F ? (size_t)(2 * upres_w1x<NU, UX>() * upres_w1y<NU>() +
                                         upres_w2x<NU, UX>() * upres_w2y<NU>()) * sizeof(float2)
                              : (size_t)upres_cw<NU, UX>() * upres_ch<NU>() * sizeof(float2);
    if constexpr (UPRES_LATE_U) return planes + (ub > planes + cs ? ub : planes + cs);
    return ub + 2 * planes + cs;
}

template <int NU, bool DAMP, int NTU, bool L1F>
__global__ void __launch_bounds__(NTU, NTU == 128 ? 7 : (UPRES_LATE_U ? 6 : 5))
k_upres2d(const InstDesc* __restrict__ insts, InstState* __restrict__ st,
          const MgItem* __restrict__ items, int e2_mode, StepCtl ctl)
{
    typedef float R;
    typedef float2 c2;
    constexpr int UX = T2;
    constexpr int TX = UX, TY = UPY;
    constexpr int NWU = NTU / 32;
    constexpr int VT = NTH / NTU;                // threads of the residual kernel's map per thread
    constexpr int H = 2 * NU + 1;
    constexpr int W = TX + 2 * H, HH = TY + 2 * H;
    constexpr int CW = upres_cw<NU, UX>(), CH = upres_ch<NU>();
    constexpr int UW = TX + 2, UH = TY + 2;
    static_assert(H % 2 == 1 && TX % 2 == 0 && TY % 2 == 0, "gx0, gy0 even");
    typedef Planes<W> PL;
    static_assert(TY == T2Y && NTH % NTU == 0, "one residual tile, NTH / NTU map threads per thread");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double sa[NTH / 32], sm[NTH / 32];
    __shared__ int last;
    // work item and descriptors are host-written: read them before the wait
    const MgItem item = items[blockIdx.y];
    const InstDesc& I = insts[item.inst];
    const LevelDesc L = I.lev[0];
    const LevelDesc C = I.lev[1];
    pdl_wait();
    pdl_trigger();
    InstState* stp = st + item.inst;
    const InstState sv = *stp;
    if (sv.status != HELM_ST_ACTIVE) {           // uniform over the CTA
        if (ctl.ctrl && blockIdx.x == 0) step_arrive(st, ctl);
        return;
    }
    const int n = L.n;
    const int ntx = (n + TX - 1) / TX;
    if ((int)blockIdx.x >= ntx * ((n + TY - 1) / TY)) return;
    const int bx = blockIdx.x % ntx, by = blockIdx.x / ntx;
    const int x0 = 1 + bx * TX, y0 = 1 + by * TY;
    constexpr int PS = HH * PL::WH;
    // early u: [U][E0 E1 R0 R1 Cs]; late u: [E0 E1][R0 R1 Cs, later U]
    double2* const U = UPRES_LATE_U
        ? reinterpret_cast<double2*>(smem_raw + (size_t)2 * PS * sizeof(c2))
        : reinterpret_cast<double2*>(smem_raw);
    c2* const base = UPRES_LATE_U ? reinterpret_cast<c2*>(smem_raw)
                                  : reinterpret_cast<c2*>(smem_raw + (size_t)UW * UH * sizeof(double2));
    c2* const E0 = base;
    c2* const E1 = base + PS;
    c2* const R0 = base + 2 * PS;
    c2* const R1 = base + 3 * PS;
    c2* const Cs = base + 4 * PS;
    const int gx0 = x0 - H, gy0 = y0 - H;
    const int cpar = (gx0 + gy0) & 1;
    const int cx0 = max(gx0, 0) >> 1, cy0 = max(gy0, 0) >> 1;
    const int nc1 = C.n + 1;
    const c2* __restrict__ gce = (const c2*)C.e;
    const int PC = C.pitch;
    const c2* __restrict__ ge2 = (const c2*)L.e2;
    const c2* __restrict__ gr = (const c2*)lev_rhs(L, 0, sv.it);
    const int P = L.pitch;
    const int S = n + 2;
    const double2* __restrict__ uin = I.u[sv.it & 1];
    const int lane = threadIdx.x & 31;
    const bool e2z = (e2_mode == 2);             // e2 zero on every level, level 0 included
    // stage u_N on the tile plus a 1-node ring (now, or after the sweeps), the coarse
    // window, e2 and r_N
    auto stage_u = [&]() {
        for (int q = threadIdx.x; q < UW * UH; q += NTU) {
            const int gx = x0 - 1 + q % UW, gy = y0 - 1 + q / UW;
            const bool in = gx <= n + 1 && gy <= n + 1;
            cp_async_elem<16>(U + q, uin + (in ? (size_t)gy * S + gx : 0), in);
        }
    };
    if (!UPRES_LATE_U) stage_u();
    // level 1 fused: its window W1 (origin c1x0, c1y0 = the coarse window's minus 2 nu2),
    // level 2's iterate under it (origin c1 >> 1) and level 1's rhs; level 1's iterate is
    // zero before its prolongation (no pre-smoothing), and its window starts cleared so that
    // the walls and the unassigned outer nodes read zero
    constexpr int W1X = upres_w1x<NU, UX>(), W1Y = upres_w1y<NU>();
    constexpr int W2X = upres_w2x<NU, UX>(), W2Y = upres_w2y<NU>();
    c2* const E1w = Cs;
    c2* const R1w = Cs + W1X * W1Y;
    c2* const C2w = Cs + 2 * W1X * W1Y;
    const int c1x0 = cx0 - 2 * NU, c1y0 = cy0 - 2 * NU;
    const int c2x0 = c1x0 >> 1, c2y0 = c1y0 >> 1;          // floor
    if constexpr (L1F) {
        const LevelDesc C2l = I.lev[2];
        const c2* __restrict__ g2e = (const c2*)C2l.e;
        const c2* __restrict__ g1r = (const c2*)C.rhs;
        const int n1 = C.n, n2 = C2l.n, P2 = C2l.pitch;
        for (int q = threadIdx.x; q < W2X * W2Y; q += NTU) {
            const int X = c2x0 + q % W2X, Y = c2y0 + q / W2X;
            const bool in = X >= 0 && X <= n2 + 1 && Y >= 0 && Y <= n2 + 1;
            cp_async_elem<sizeof(c2)>(C2w + q, g2e + (in ? (size_t)Y * P2 + X : 0), in);
        }
        for (int q = threadIdx.x; q < W1X * W1Y; q += NTU) {
            const int X = c1x0 + q % W1X, Y = c1y0 + q / W1X;
            const bool in = X >= 1 && X <= n1 && Y >= 1 && Y <= n1;
            cp_async_elem<sizeof(c2)>(R1w + q, g1r + (in ? (size_t)Y * PC + X : 0), in);
            E1w[q] = cz<c2>();
        }
        // level 1's words form the first group of copies: its ascent starts on them while
        // level 0's window is still arriving
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    } else {
        for (int q = threadIdx.x; q < CW * CH; q += NTU) {
            const int cy = q / CW, cx = q - cy * CW;
            const int X = cx0 + cx, Y = cy0 + cy;
            const bool in = X <= nc1 && Y <= nc1;
            cp_async_elem<sizeof(c2)>(Cs + q, gce + (in ? (size_t)Y * PC + X : 0), in);
        }
    }
    // the window's W x HH nodes numbered row by row over the threads (rows of a few dozen
    // nodes: a warp per row would leave lanes idle)
    for (int q = threadIdx.x; q < W * HH; q += NTU) {
        const int ly = q / W, lx = q - ly * W;
        const int gy = gy0 + ly;
        const bool yin = gy >= 1 && gy <= n;
        const int gx = gx0 + lx;
        const bool in = yin && gx >= 1 && gx <= n;
        const size_t g = in ? (size_t)gy * P + gx : 0;
        const int c = (lx + ly + cpar) & 1;
        const int o = PL::at(lx, ly);
        // with post-smoothing the first half-sweep overwrites every interior colour-0
        // node it reads later, without reading their old values: colour 0 needs e2
        // only off the interior (the walls' zeros, which the sweeps read)
        if (NU == 0 || c || !in) {
            if (e2z) (c ? E1 : E0)[o] = cz<c2>();
            else cp_async_elem<sizeof(c2)>((c ? E1 : E0) + o, ge2 + g, in);
        }
        cp_async_elem<sizeof(c2)>((c ? R1 : R0) + o, gr + g, in);
    }
    if constexpr (L1F) {
        asm volatile("cp.async.commit_group;\n" ::: "memory");
        asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    } else {
        cp_async_wait_all();
    }
    __syncthreads();
    if constexpr (L1F) {
        // level 1's ascent on the window, as k_up2d forms it: e := 0 + the interpolation of
        // level 2 (colour 1 only when sweeps follow: the first half-sweep overwrites colour 0
        // without reading it), then nu2 sweeps, each half-sweep one node closer to the coarse
        // window, whose values end final
        const int n1 = C.n;
        for (int q = threadIdx.x; q < W1X * W1Y; q += NTU) {
            const int i = q % W1X, j = q / W1X;
            const int X = c1x0 + i, Y = c1y0 + j;
            if (X < 1 || X > n1 || Y < 1 || Y > n1) continue;
            if (NU > 0 && ((X + Y) & 1) == 0) continue;
            const int X0 = (X >> 1) - c2x0, X1 = ((X + 1) >> 1) - c2x0;
            const int Y0 = (Y >> 1) - c2y0, Y1 = ((Y + 1) >> 1) - c2y0;
            const c2 a = C2w[Y0 * W2X + X0], b = C2w[Y0 * W2X + X1];
            const c2 c = C2w[Y1 * W2X + X0], d = C2w[Y1 * W2X + X1];
            c2 v;
            v.x = (R)0 + (R)0.25 * (((a.x + b.x) + c.x) + d.x);
            v.y = (R)0 + (R)0.25 * (((a.y + b.y) + c.y) + d.y);
            E1w[q] = v;
        }
        __syncthreads();
        const R h21 = (R)(C.h * C.h);
        const R dinv1 = (R)C.dinv;
#pragma unroll 1
        for (int sw = 1; sw <= 2 * NU; ++sw) {
            const int color = (sw - 1) & 1, ring1 = 2 * NU - sw;
            const int xa = max(cx0 - ring1, 1), xb = min(cx0 + CW - 1 + ring1, n1);
            const int ya = max(cy0 - ring1, 1), yb = min(cy0 + CH - 1 + ring1, n1);
            for (int Y = ya + (int)(threadIdx.x >> 5); Y <= yb; Y += NWU) {
                const int xs = xa + (((xa + Y) & 1) ^ color);
                const int j = Y - c1y0;
                for (int X = xs + 2 * lane; X <= xb; X += 64) {
                    const int o1 = j * W1X + (X - c1x0);
                    const c2 a = E1w[o1 - 1], b = E1w[o1 + 1], c = E1w[o1 - W1X], d = E1w[o1 + W1X];
                    const c2 rr = R1w[o1];
                    c2 v;
                    v.x = ((a.x + b.x + c.x + d.x) - h21 * rr.x) * dinv1;
                    v.y = ((a.y + b.y + c.y + d.y) - h21 * rr.y) * dinv1;
                    E1w[o1] = v;
                }
            }
            __syncthreads();
        }
        cp_async_wait_all();                     // level 0's window
        __syncthreads();
    }
    // level 1's final iterate on the coarse window (its own buffer, or the fused window's
    // centre)
    constexpr int CSTR = L1F ? W1X : CW;
    const c2* const Cr = L1F ? E1w + 2 * NU * W1X + 2 * NU : Cs;
    // correction: e2 + multilinear interpolation of the coarse iterate (interior nodes);
    // with post-smoothing only on colour 1 (the first half-sweep overwrites colour 0, and
    // the outermost ring's colour-0 nodes it leaves are never read)
    // nodes numbered row by row over the threads: all W of a row, or its W / 2 colour-1 nodes
    constexpr int CNX = (NU == 0) ? W : W / 2;
    for (int q = threadIdx.x; q < CNX * HH; q += NTU) {
        const int ly = q / CNX, i = q - ly * CNX;
        const int gy = gy0 + ly;
        if (gy < 1 || gy > n) continue;
        const int Y0 = (gy >> 1) - cy0, Y1 = ((gy + 1) >> 1) - cy0;
        const int lx = (NU == 0) ? i : 2 * i + ((ly + cpar + 1) & 1);
        const int gx = gx0 + lx;
        if (gx < 1 || gx > n) continue;
        const int X0 = (gx >> 1) - cx0, X1 = ((gx + 1) >> 1) - cx0;
        const c2 a = Cr[Y0 * CSTR + X0], b = Cr[Y0 * CSTR + X1];
        const c2 c = Cr[Y1 * CSTR + X0], d = Cr[Y1 * CSTR + X1];
        c2* Ep = (((lx + ly + cpar) & 1) ? E1 : E0) + PL::at(lx, ly);
        c2 v = *Ep;
        v.x += (R)0.25 * (((a.x + b.x) + c.x) + d.x);
        v.y += (R)0.25 * (((a.y + b.y) + c.y) + d.y);
        *Ep = v;
    }
    __syncthreads();
    const R h2 = (R)(L.h * L.h);
    const R dinv = (R)L.dinv;
    sweeps_flat<R, W, TX, TY, NTU, 2 * NU, 2 * NU>(E0, E1, R0, R1, gx0, gy0, x0, y0, n, h2, dinv);
    if (UPRES_LATE_U) {                          // the rhs planes and Cs are dead: u_N there
        stage_u();
        cp_async_wait_all();
        __syncthreads();
    }
    // u_{N+1} = u_N + e_N on the window (as k_residual2d forms it): the residual nodes of
    // each map thread in registers, the ring by the first threads; the window's largest
    // exponent sets the scale of the exact fixed-point Laplacian numerators
    constexpr int KY = TY / 8, RING = 2 * (TX + 2) + 2 * TY, RJ = (RING + NTU - 1) / NTU;
    __shared__ int sx[NWU];
    double2 cv[VT][KY];
    int exq = 0;
    // window node (lxw, lyw): u_N (+ e_N inside the grid; |e_N|^2 into *em for own nodes)
    auto upd = [&](int lxw, int lyw, R* em) -> double2 {
        const int gx = x0 - 1 + lxw, gy = y0 - 1 + lyw;
        double2 v = U[lyw * UW + lxw];
        if (gx >= 1 && gx <= n && gy >= 1 && gy <= n) {
            const int ex = gx - gx0, ey = gy - gy0;
            const c2 ev = (((ex + ey + cpar) & 1) ? E1 : E0)[PL::at(ex, ey)];
            v.x += Inner<R>::widen(ev.x);
            v.y += Inner<R>::widen(ev.y);
            if (em) *em = fmax(*em, abs2(ev));
        }
        return v;
    };
    R r2[VT], em[VT];
#pragma unroll
    for (int v = 0; v < VT; ++v) {
        const int t = threadIdx.x + NTU * v;
        em[v] = 0;
#pragma unroll
        for (int k = 0; k < KY; ++k) {
            cv[v][k] = upd((t & 31) + 1, (t >> 5) + 8 * k + 1, &em[v]);
            exq = max(exq, fx_exp2(cv[v][k]));
        }
    }
    double2 rv[RJ];
    int rq[RJ];
#pragma unroll
    for (int j = 0; j < RJ; ++j) {
        const int t = threadIdx.x + NTU * j;
        rq[j] = -1;
        rv[j] = make_double2(0.0, 0.0);
        if (t < RING) {
            int rlx, rly;
            ring_node<TX, TY>(t, rlx, rly);
            rv[j] = upd(rlx, rly, nullptr);
            rq[j] = rly * UW + rlx;
            exq = max(exq, fx_exp2(rv[j]));
        }
    }
    // its barrier also ends the reads of U; uniform over the CTA
    const int emx = fx_scale(block_max_exp<NTU>(exq, sx));
    longlong2* UF = reinterpret_cast<longlong2*>(U);
#pragma unroll
    for (int v = 0; v < VT; ++v) {
        const int t = threadIdx.x + NTU * v;
#pragma unroll
        for (int k = 0; k < KY; ++k) UF[((t >> 5) + 8 * k + 1) * UW + (t & 31) + 1] = fx_fix2(cv[v][k], emx);
    }
#pragma unroll
    for (int j = 0; j < RJ; ++j)
        if (rq[j] >= 0) UF[rq[j]] = fx_fix2(rv[j], emx);
    __syncthreads();
    // r_{N+1}: thread t of the residual kernel's map takes the nodes (t mod 32, t / 32 + 8 k)
    // of the tile; real thread j stands for the map's threads j + NTU v, v < VT
    double2* __restrict__ uout = I.u[(sv.it + 1) & 1];
    c2* __restrict__ rhs = (c2*)lev_rhs(L, 0, sv.it + 1);
    const double2* __restrict__ f = I.f;
    const double mih2 = -I.ih2, mk2 = -I.k2;
    const double damp = I.damp;
#pragma unroll
    for (int v = 0; v < VT; ++v) {
        const int t = threadIdx.x + NTU * v;
        const int lx = (t & 31) + 1;
        r2[v] = 0;
#pragma unroll
        for (int k = 0; k < TY / 8; ++k) {
            const int ly = (t >> 5) + 8 * k + 1;
            const int gx = x0 + lx - 1, gy = y0 + ly - 1;
            if (gx > n || gy > n) continue;
            const int o = ly * UW + lx;
            const double2 c = cv[v][k];
            uout[(size_t)gy * S + gx] = c;
            const double2 fv = f[(size_t)(gy - 1) * n + (gx - 1)];
            const double2 r = (emx >= 0)
                ? helm_resid2d_fx<DAMP>(c, UF[o], UF[o - 1], UF[o + 1], UF[o - UW], UF[o + UW], fv, mih2, mk2,
                                        damp, emx)
                : make_double2(fx_nan(), fx_nan());
            const c2 ri = Inner<R>::from(r);
            rhs[(size_t)gy * P + gx] = ri;
            r2[v] += abs2(ri);
        }
    }
    // the tile's partials in k_residual2d's order, then the instance's ticket
    double ra = 0.0, rm = 0.0;
    block_reduce_v<R, VT>(r2, em, ra, rm, sa, sm, false);
    const int nb = I.nres_blocks;
    if (threadIdx.x == 0) {
        const int tile = by * I.res_tx + bx;
        I.part[tile] = ra;
        I.part[nb + tile] = rm;
        __threadfence();
        last = (atomicAdd(I.count, 1u) == (unsigned)(nb - 1));
    }
    __syncthreads();
    if (!last) return;
    instance_last<VT>(I, stp, 1, st, ctl, sa, sm);
}

// ---------------------------------------------------------------------------
// 3D: 32 x 8 columns marching over 16 z-planes; u_{N+1} staged once per node in a
// three-plane ring of shared memory (1-node halo in x and y)
// ---------------------------------------------------------------------------
constexpr int T3X = 32, T3Y = 8, T3Z = 16;
// resident CTAs per SM of the 3D residual (40 registers at 6): at 255^3 477 -> 396 us per
// launch against 4 CTAs of 64 registers; fetching each plane one plane ahead into
// registers measured slower (412 / 432 / 485 us at 4 / 5 / 6 CTAs), and so did a two-deep
// cp.async ring of the next planes' words in shared memory (425 against 385 us: 5 CTAs
// per SM, and the copies' issue cost on a kernel bound by its integer work)
constexpr int RES3D_CTAS = 6;
constexpr int P3 = (T3X + 2) * (T3Y + 2);

// The column's planes go through the ring in fixed point
// (fixed_lap.cuh), each plane on the scale of its own largest exponent; the numerator of
// plane z is summed on the largest scale of planes z - 1, z, z + 1 (the other planes'
// values shifted down to it), so every node's numerator is exact up to the truncations.
// Thread t stages the interior node (t mod 32, t / 32) of each plane and keeps it in FP64
// for its own residual; threads below the ring size stage one ring node each.
template <typename R, int MODE, bool DAMP>
__device__ __forceinline__ void residual3d_tile_fx(const InstDesc* __restrict__ insts,
                                                   InstState* __restrict__ st, const ResItem item,
                                                   longlong2 (*U)[P3], int* sx, const StepCtl& c)
{
    typedef typename C2<R>::T c2;
    static_assert(T3X * T3Y == NTH, "one interior node of a plane per thread");
    constexpr int RING = 2 * (T3X + 2) + 2 * T3Y;
    static_assert(RING <= NTH, "one ring node per thread");
    const InstDesc& I = insts[item.inst];
    const int n = I.n;
    const long S = n + 2;
    const long SP = S * S;
    InstState* stp = st + item.inst;
    const InstState s = *stp;
    if (s.status != HELM_ST_ACTIVE) {           // uniform over the CTA
        if (c.ctrl && item.tx == 0 && item.ty == 0 && item.tz == 0) step_arrive(st, c);
        return;
    }
    const double2* __restrict__ uin = (s.it & 1) ? I.u[1] : I.u[0];
    double2* __restrict__ uout = (double2*)((s.it & 1) ? I.u[0] : I.u[1]);
    const double2* __restrict__ f = I.f;
    const LevelDesc L0 = I.lev[0];
    const c2* __restrict__ e = (const c2*)L0.e;
    c2* __restrict__ rhs = (c2*)lev_rhs(L0, 0, MODE == 1 ? s.it + 1 : s.it);   // r_{N+1} / r_0
    const long P = L0.pitch;
    const long PL = (long)L0.pitch * L0.rows;
    const double mih2 = -I.ih2, mk2 = -I.k2;
    const double damp = I.damp;
    const int x0 = 1 + item.tx * T3X, y0 = 1 + item.ty * T3Y, z0 = 1 + item.tz * T3Z;
    const int z1 = min(z0 + T3Z - 1, n);
    const int lx = (threadIdx.x & 31) + 1, ly = (threadIdx.x >> 5) + 1;
    const int gx = x0 + lx - 1, gy = y0 + ly - 1;
    const bool live = gx <= n && gy <= n;
    const int o = ly * (T3X + 2) + lx;
    int rlx = 0, rly = 0;
    if (threadIdx.x < RING) ring_node<T3X, T3Y>(threadIdx.x, rlx, rly);
    const int ro = rly * (T3X + 2) + rlx;
    R r2 = 0, emax2 = 0;
    double r2d = 0.0, b2 = 0.0;
    // u_{N+1} at window node (wx, wy) of plane gz: u_N, plus e_N at interior nodes (mode 1;
    // mode 0 takes the iterate as it is)
    auto node = [&](int wx, int wy, int gz, bool own) -> double2 {
        const int nx = x0 - 1 + wx, ny = y0 - 1 + wy;
        double2 v = make_double2(0.0, 0.0);
        if (nx <= n + 1 && ny <= n + 1 && gz <= n + 1) {
            v = uin[(long)gz * SP + (long)ny * S + nx];
            if (MODE == 1 && nx >= 1 && nx <= n && ny >= 1 && ny <= n && gz >= 1 && gz <= n) {
                const c2 ev = e[(long)gz * PL + (long)ny * P + xslot<3>(nx, (int)P)];
                v.x += Inner<R>::widen(ev.x);
                v.y += Inner<R>::widen(ev.y);
                if (own) emax2 = fmax(emax2, abs2(ev));
            }
        }
        return v;
    };
    // stage plane gz into ring slot `slot`: returns its scale exponent (-1: none); the
    // thread's own node in FP64 goes to `mine`
    auto stage = [&](int slot, int gz, bool own, double2& mine) -> int {
        mine = node(lx, ly, gz, own && live);
        double2 rv = make_double2(0.0, 0.0);
        if (threadIdx.x < RING) rv = node(rlx, rly, gz, false);
        const int ep = fx_scale(block_max_exp<NTH>(max(fx_exp2(mine), fx_exp2(rv)), sx));
        U[slot][o] = fx_fix2(mine, ep);
        if (threadIdx.x < RING) U[slot][ro] = fx_fix2(rv, ep);
        return ep;
    };
    int ep[3];
    double2 cur, nxt, dummy;
    ep[0] = stage(0, z0 - 1, false, dummy);
    __syncthreads();                            // sx is reused by the next stage
    ep[1] = stage(1, z0, true, cur);
    int sp = 0, sc = 1, sn = 2;                 // ring slots of planes z-1, z, z+1
    for (int z = z0; z <= z1; ++z) {
        // no barrier needed here: stage writes sx before, and the oldest slot after, the
        // barrier inside its exponent reduction, which every thread reaches only once done
        // with the previous plane (its reads of sx and of that slot)
        ep[sn] = stage(sn, z + 1, z + 1 <= z1, nxt);
        __syncthreads();
        if (live) {
            const int em = max(max(ep[sp], ep[sc]), ep[sn]);
            double2 r;
            if (ep[sp] >= 0 && ep[sc] >= 0 && ep[sn] >= 0) {
                // shifts to the common scale (arithmetic, so each rounds toward -inf once);
                // |in-plane part| < 10 * 2^58 and the total < 12 * 2^58 < 2^62
                const int dc = min(em - ep[sc], 63), dd = min(em - ep[sp], 63), du = min(em - ep[sn], 63);
                const longlong2* Uc = U[sc];
                const longlong2 C = Uc[o], W = Uc[o - 1], E = Uc[o + 1];
                const longlong2 So = Uc[o - (T3X + 2)], No = Uc[o + (T3X + 2)];
                const longlong2 Dn = U[sp][o], Up = U[sn][o];
                const long long lx_ = ((((W.x + E.x) + (So.x + No.x)) - 6 * C.x) >> dc) + ((Dn.x >> dd) + (Up.x >> du));
                const long long ly_ = ((((W.y + E.y) + (So.y + No.y)) - 6 * C.y) >> dc) + ((Dn.y >> dd) + (Up.y >> du));
                const double2 fv = f[((long)(z - 1) * n + (gy - 1)) * n + (gx - 1)];
                r = helm_resid_fx<DAMP>(cur, lx_, ly_, fv, mih2, mk2, damp, em);
                if (MODE == 0) {
                    // once per solve, in FP64: ||r_0||^2 and ||b||^2, b = f - (wall
                    // neighbours) / h^2, formed with r's operations (r_0 = b bit for bit from
                    // a zero start: its numerator then holds the wall values alone)
                    r2d += r.x * r.x + r.y * r.y;
                    double bx = fv.x, by = fv.y;
                    if (gx == 1 || gx == n || gy == 1 || gy == n || z == 1 || z == n) {
                        const longlong2 zz = make_longlong2(0, 0);
                        const longlong2 w1 = (gx == 1) ? W : zz, w2 = (gx == n) ? E : zz;
                        const longlong2 w3 = (gy == 1) ? So : zz, w4 = (gy == n) ? No : zz;
                        const longlong2 w5 = (z == 1) ? Dn : zz, w6 = (z == n) ? Up : zz;
                        const long long bx_ = ((((w1.x + w2.x) + (w3.x + w4.x)) - 6 * zz.x) >> dc) + ((w5.x >> dd) + (w6.x >> du));
                        const long long by_ = ((((w1.y + w2.y) + (w3.y + w4.y)) - 6 * zz.y) >> dc) + ((w5.y >> dd) + (w6.y >> du));
                        const double2 bb = helm_resid_fx<false>(make_double2(0.0, 0.0), bx_, by_, fv, mih2, mk2, 0.0, em);
                        bx = bb.x;
                        by = bb.y;
                    }
                    b2 += bx * bx + by * by;
                }
            } else {
                r = make_double2(fx_nan(), fx_nan());
                if (MODE == 0) r2d += r.x;
            }
            if (MODE == 1) uout[(long)z * SP + (long)gy * S + gx] = cur;
            const c2 ri = Inner<R>::from(r);
            rhs[(long)z * PL + (long)gy * P + xslot<3>(gx, (int)P)] = ri;
            if (MODE == 1) r2 += abs2(ri);
        }
        cur = nxt;
        const int t = sp;
        sp = sc;
        sc = sn;
        sn = t;
    }
    const int tile = (item.tz * I.res_ty + item.ty) * I.res_tx + item.tx;
    if constexpr (MODE == 0) tile_done<double>(I, stp, tile, r2d, b2, MODE, st, c);
    else tile_done<R>(I, stp, tile, r2, emax2, MODE, st, c);
}

// (the start residual, once per solve, also forms ||b||: it runs at 4 CTAs per SM, whose 64
// registers cut its spills from 260 to 88 bytes)
template <typename R, int MODE, bool DAMP>
__global__ void __launch_bounds__(NTH, MODE == 1 ? RES3D_CTAS : 4)
k_residual3d(const InstDesc* __restrict__ insts, InstState* __restrict__ st,
             const ResItem* __restrict__ items, int nitems, StepCtl c)
{
    __shared__ double2 U[3][P3];
    __shared__ int sx[NTH / 32];
    pdl_wait();
    pdl_trigger();
    for (int t = blockIdx.x; t < nitems; t += gridDim.x) {
        residual3d_tile_fx<R, MODE, DAMP>(insts, st, items[t], reinterpret_cast<longlong2(*)[P3]>(U), sx, c);
        __syncthreads();
    }
}

// One CTA: the step control when it is not folded into the residual launch.
__global__ void __launch_bounds__(256)
k_check(const InstState* __restrict__ st, int ninst, int* __restrict__ ctrl, int use_cond,
        unsigned long long cond_handle)
{
    pdl_wait();
    pdl_trigger();
    step_end(st, ninst, ctrl, use_cond, cond_handle);
}

template <int D>
__global__ void k_set_ring(const InstDesc* __restrict__ insts, int inst)
{
    pdl_wait();
    pdl_trigger();
    const InstDesc& I = insts[inst];
    const int n = I.n, S = n + 2;
    const long total = (D == 3) ? (long)S * S * S : (long)S * S;
    for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < total;
         q += (long)gridDim.x * blockDim.x) {
        const int x = (int)(q % S);
        const int y = (int)((q / S) % S);
        const int z = (D == 3) ? (int)(q / ((long)S * S)) : 1;
        const bool ring = x == 0 || x == S - 1 || y == 0 || y == S - 1 ||
                          (D == 3 && (z == 0 || z == S - 1));
        if (ring) {
            const double2 v = I.g[q];
            I.u[0][q] = v;
            I.u[1][q] = v;
        }
    }
}

// k_set_ring for several instances of one size: instance slots[blockIdx.y]
template <int D>
__global__ void k_set_ring_many(const InstDesc* __restrict__ insts, const int* __restrict__ slots)
{
    pdl_wait();
    pdl_trigger();
    const InstDesc& I = insts[slots[blockIdx.y]];
    const int n = I.n, S = n + 2;
    const long total = (D == 3) ? (long)S * S * S : (long)S * S;
    for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < total;
         q += (long)gridDim.x * blockDim.x) {
        const int x = (int)(q % S);
        const int y = (int)((q / S) % S);
        const int z = (D == 3) ? (int)(q / ((long)S * S)) : 1;
        const bool ring = x == 0 || x == S - 1 || y == 0 || y == S - 1 ||
                          (D == 3 && (z == 0 || z == S - 1));
        if (ring) {
            const double2 v = I.g[q];
            I.u[0][q] = v;
            I.u[1][q] = v;
        }
    }
}

// the residual tiles of instances slots[0 .. m): T = tx * ty * tz tiles each, in order
__global__ void k_fill_res_many(ResItem* __restrict__ items, const int* __restrict__ slots, int tx, int ty,
                                int T, int total)
{
    pdl_wait();
    pdl_trigger();
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < total; q += gridDim.x * blockDim.x) {
        const int j = q / T, t = q - j * T;
        items[q] = ResItem{slots[j], t % tx, (t / tx) % ty, t / (tx * ty)};
    }
}

template <int D, typename R>
__global__ void k_pack(const InstDesc* __restrict__ insts, int inst, const void* __restrict__ src,
                       int which)
{
    pdl_wait();
    pdl_trigger();
    typedef typename C2<R>::T c2;
    const InstDesc& I = insts[inst];
    const LevelDesc L = I.lev[0];
    const int n = L.n;
    const long total = (D == 3) ? (long)n * n * n : (long)n * n;
    c2* dst = (c2*)(which ? L.rhs : L.e);
    const c2* s = (const c2*)src;
    for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < total;
         q += (long)gridDim.x * blockDim.x) {
        const int x = (int)(q % n) + 1;
        const int y = (int)((q / n) % n) + 1;
        const int z = (D == 3) ? (int)(q / ((long)n * n)) + 1 : 0;
        dst[((D == 3) ? ((long)z * L.rows + y) : (long)y) * L.pitch + xslot<D>(x, L.pitch)] = s[q];
    }
}

template <int D, typename R>
__global__ void k_unpack(const InstDesc* __restrict__ insts, int inst, void* __restrict__ dst)
{
    pdl_wait();
    pdl_trigger();
    typedef typename C2<R>::T c2;
    const InstDesc& I = insts[inst];
    const LevelDesc L = I.lev[0];
    const int n = L.n;
    const long total = (D == 3) ? (long)n * n * n : (long)n * n;
    const c2* src = (const c2*)L.e;
    c2* d = (c2*)dst;
    for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < total;
         q += (long)gridDim.x * blockDim.x) {
        const int x = (int)(q % n) + 1;
        const int y = (int)((q / n) % n) + 1;
        const int z = (D == 3) ? (int)(q / ((long)n * n)) + 1 : 0;
        d[q] = src[((D == 3) ? ((long)z * L.rows + y) : (long)y) * L.pitch + xslot<D>(x, L.pitch)];
    }
}

// Mean exit time support (Eq. (2.10)): the constant source, and max Re(u) over the interior
// of a padded array, clamped at 0 (E >= 0): block maxima, then an atomic maximum on the bit
// patterns (non-negative doubles order as their bits), so the result is exact and order-free.
__global__ void k_fill_c128(double2* __restrict__ p, long count, double re, double im)
{
    pdl_wait();
    pdl_trigger();
    for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < count; q += (long)gridDim.x * blockDim.x)
        p[q] = make_double2(re, im);
}

template <int D>
__global__ void __launch_bounds__(256)
k_max_re(const double2* __restrict__ u, int n, unsigned long long* __restrict__ out)
{
    pdl_wait();
    pdl_trigger();
    const long S = n + 2;
    const long total = (D == 3) ? (long)n * n * n : (long)n * n;
    double m = 0.0;
    for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < total; q += (long)gridDim.x * blockDim.x) {
        const long x = q % n + 1, y = (q / n) % n + 1, z = (D == 3) ? q / ((long)n * n) + 1 : 0;
        const double v = u[((D == 3) ? (z * S + y) : y) * S + x].x;
        m = fmax(m, v);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    __shared__ double sw[8];
    if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) b = fmax(b, sw[i]);
        atomicMax(out, (unsigned long long)__double_as_longlong(b));
    }
}

// Power iteration support on the finest level's arrays (interior nodes only; the rings
// stay zero): fill, sum of squares (fixed-order block partials, then one block in order),
// rhs = s * e.
constexpr int PI_BLOCKS = 512;

template <int D>
__device__ __forceinline__ long lev_off(const LevelDesc& L, long q)
{
    const int n = L.n;
    const long x = q % n + 1, y = (q / n) % n + 1, z = (D == 3) ? q / ((long)n * n) + 1 : 0;
    return ((D == 3) ? (z * L.rows + y) : y) * (long)L.pitch + xslot<D>((int)x, L.pitch);
}

template <int D, typename R>
__global__ void k_lev_fill(const InstDesc* __restrict__ insts, int which, double re)
{
    pdl_wait();
    pdl_trigger();
    typedef typename C2<R>::T c2;
    const LevelDesc L = insts[0].lev[0];
    c2* a = (c2*)(which ? L.rhs : L.e);
    const long total = (D == 3) ? (long)L.n * L.n * L.n : (long)L.n * L.n;
    c2 v;
    v.x = (R)re;
    v.y = (R)0;
    for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < total; q += (long)gridDim.x * blockDim.x)
        a[lev_off<D>(L, q)] = v;
}

template <int D, typename R>
__global__ void __launch_bounds__(256)
k_lev_sumsq(const InstDesc* __restrict__ insts, double* __restrict__ partial)
{
    pdl_wait();
    pdl_trigger();
    typedef typename C2<R>::T c2;
    const LevelDesc L = insts[0].lev[0];
    const c2* a = (const c2*)L.e;
    const long total = (D == 3) ? (long)L.n * L.n * L.n : (long)L.n * L.n;
    double acc = 0.0;
    for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < total; q += (long)gridDim.x * blockDim.x) {
        const c2 v = a[lev_off<D>(L, q)];
        acc += (double)v.x * (double)v.x + (double)v.y * (double)v.y;
    }
    __shared__ double sa[8], sm[8];
    double m = 0.0, ra = 0.0, rm = 0.0;
    block_reduce<double>(acc, m, ra, rm, sa, sm, true);
    if (threadIdx.x == 0) partial[blockIdx.x] = ra;
}

__global__ void k_sum_partials(const double* __restrict__ partial, int nb, double* __restrict__ out)
{
    pdl_wait();
    pdl_trigger();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < nb; ++i) s += partial[i];
        *out = s;
    }
}

template <int D, typename R>
__global__ void k_lev_scale(const InstDesc* __restrict__ insts, double sc)
{
    pdl_wait();
    pdl_trigger();
    typedef typename C2<R>::T c2;
    const LevelDesc L = insts[0].lev[0];
    const c2* e = (const c2*)L.e;
    c2* r = (c2*)L.rhs;
    const long total = (D == 3) ? (long)L.n * L.n * L.n : (long)L.n * L.n;
    for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < total; q += (long)gridDim.x * blockDim.x) {
        const long o = lev_off<D>(L, q);
        const c2 v = e[o];
        c2 w;
        w.x = (R)((double)v.x * sc);
        w.y = (R)((double)v.y * sc);
        r[o] = w;
    }
}

// Self-test of the integer-pipe conversions against the hardware conversions on random
// values of the binary32 range, exact ties, and the special values.
__device__ __forceinline__ unsigned long long splitmix(unsigned long long x)
{
    x += 0x9e3779b97f4a7c15ull;
    x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ull;
    x = (x ^ (x >> 27)) * 0x94d049bb133111ebull;
    return x ^ (x >> 31);
}

__global__ void k_fp_bits_check(unsigned long long seed, int count, unsigned long long* bad)
{
    unsigned long long local = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        const unsigned long long r = splitmix(seed + (unsigned long long)i);
        // binary64 with an exponent inside (or just outside) the binary32 range
        const unsigned long long ex = 1023ull - 130ull + ((r >> 52) % 261ull);
        unsigned long long frac = r & 0x000fffffffffffffull;
        const unsigned kind = (unsigned)(r >> 61);
        if (kind == 0) frac = (frac & ~0x1fffffffull) | 0x10000000ull;   // exact tie
        if (kind == 1) frac &= ~0x1fffffffull;                           // exactly representable
        const unsigned long long bits = ((r >> 51) & 1ull) << 63 | ex << 52 | frac;
        double d = __longlong_as_double((long long)bits);
        if (i < 6) {
            const double sp[6] = {0.0, -0.0, 1.0 / 0.0, -1.0 / 0.0, 0.0 / 0.0, 3.4028235677973366e38};
            d = sp[i];
        }
        const float ref = __double2float_rn(d);
        const float got = d2f_bits(d);
        const unsigned rb = __float_as_uint(ref), gb = __float_as_uint(got);
        const bool sub = (rb & 0x7f800000u) == 0u && (rb & 0x007fffffu) != 0u;
        if (!sub && !(isnan(ref) && isnan(got)) && rb != gb) ++local;
        // binary32 -> binary64 (exact) on the normal range and the special values
        const float f = __uint_as_float((unsigned)(r >> 17));
        const unsigned fb = __float_as_uint(f);
        const bool fsub = (fb & 0x7f800000u) == 0u && (fb & 0x007fffffu) != 0u;
        const double w = f2d_bits(f), wr = (double)f;
        if (!fsub && !(isnan(w) && isnan(wr)) && __double_as_longlong(w) != __double_as_longlong(wr)) ++local;
    }
    if (local) atomicAdd(bad, local);
}

// FP64 issue-rate probe: every thread runs 8 independent FMA chains x = x * m + c
// (m, c kernel arguments, |m| < 1, so nothing overflows or turns subnormal and the
// compiler cannot fold the loop); the sum of the chains is stored so no chain is dead.
__global__ void __launch_bounds__(256) k_fp64_rate(int iters, double m, double c, double* sink)
{
    double x[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = 1.0 + 1e-3 * (threadIdx.x + j);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < 8; ++j) x[j] = fma(x[j], m, c);
    }
    double t = 0.0;
#pragma unroll
    for (int j = 0; j < 8; ++j) t += x[j];
    if (t == 12345.678) sink[blockIdx.x * blockDim.x + threadIdx.x] = t;   // never true
}

inline int blocks_for(long work) {
    long b = (work + 255) / 256;
    if (b < 1) b = 1;
    if (b > 2432) b = 2432;
    return (int)b;
}

}  // namespace

int residual_tile_rows(int D) { return D == 2 ? T2Y : T3Y; }
int residual_tile_planes(int D) { return D == 2 ? 1 : T3Z; }

cudaError_t run_fp_bits_check(int count, unsigned long long seed, unsigned long long* bad_host)
{
    unsigned long long* d = nullptr;
    cudaError_t e = cudaMalloc(&d, sizeof(unsigned long long));
    if (e != cudaSuccess) return e;
    cudaMemset(d, 0, sizeof(unsigned long long));
    k_fp_bits_check<<<1216, 256>>>(seed, count, d);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpy(bad_host, d, sizeof(unsigned long long), cudaMemcpyDeviceToHost);
    cudaFree(d);
    return e;
}
int residual_tile_cols(int D) { return 32; }

namespace {
__global__ void k_fill_res_items(ResItem* __restrict__ items, int tx, int ty, int total)
{
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < total; q += gridDim.x * blockDim.x)
        items[q] = ResItem{0, q % tx, (q / tx) % ty, q / (tx * ty)};
}

// blockIdx.y = record; the record's blocks stride over its 16-byte words (then the bytes
// of a ragged end) and its tile list
__global__ void __launch_bounds__(256) k_init_ws(const WsInit* __restrict__ recs)
{
    const WsInit r = recs[blockIdx.y];
    const unsigned long long n16 = r.bytes >> 4;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    const unsigned long long t0 = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    uint4* w = reinterpret_cast<uint4*>(r.ws);
    for (unsigned long long q = t0; q < n16; q += stride) w[q] = make_uint4(0u, 0u, 0u, 0u);
    for (unsigned long long q = (n16 << 4) + t0; q < r.bytes; q += stride) r.ws[q] = 0;
    const unsigned long long total = (unsigned long long)r.tx * r.ty * r.tz;
    for (unsigned long long q = t0; q < total; q += stride) {
        const int qi = (int)q;
        r.items[qi] = ResItem{0, qi % r.tx, (qi / r.tx) % r.ty, qi / (r.tx * r.ty)};
    }
}
}  // namespace

cudaError_t launch_init_workspaces(const WsInit* recs, int count, cudaStream_t s)
{
    for (int off = 0; off < count; off += 65535) {
        const int m = count - off < 65535 ? count - off : 65535;
        k_init_ws<<<dim3(128, m), 256, 0, s>>>(recs + off);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_fill_res_items(ResItem* items, int tx, int ty, int tz, cudaStream_t s)
{
    const int total = tx * ty * tz;
    if (total <= 0) return cudaSuccess;
    k_fill_res_items<<<(total + 255) / 256 < 1024 ? (total + 255) / 256 : 1024, 256, 0, s>>>(items, tx, ty, total);
    return cudaGetLastError();
}

cudaError_t run_fp64_rate(double* tflops, double* ms_best)
{
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int blocks = sms * 8, threads = 256, iters = 4096;
    double* sink = nullptr;
    e = cudaMalloc(&sink, sizeof(double) * blocks * threads);
    if (e != cudaSuccess) return e;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    float best = 1e30f;
    for (int rep = 0; rep < 6 && e == cudaSuccess; ++rep) {
        cudaEventRecord(a, 0);
        k_fp64_rate<<<blocks, threads>>>(iters, 0.9999999, 1e-7, sink);
        cudaEventRecord(b, 0);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventSynchronize(b);
        float t = 0.0f;
        if (e == cudaSuccess) cudaEventElapsedTime(&t, a, b);
        if (rep > 0 && t > 0.0f && t < best) best = t;        // the first launch warms up
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(sink);
    if (e != cudaSuccess) return e;
    const double flops = 2.0 * 8.0 * (double)iters * blocks * threads;
    *ms_best = best;
    *tflops = flops / (best * 1e-3) / 1e12;
    return cudaSuccess;
}

cudaError_t launch_residual(int D, int prec, const InstDesc* insts, InstState* st,
                            const ResItem* items, int nitems, int mode, cudaStream_t s,
                            int* ctrl, int nscan, int ninst, int use_cond,
                            unsigned long long cond_handle, int damp)
{
    if (nitems <= 0) return cudaSuccess;
    const StepCtl c{ctrl, nscan, ninst, use_cond, cond_handle};
    // one CTA per tile: measured faster than a persistent grid (SMs x resident CTAs
    // striding over the tiles) for both the 2D tiles and the 3D columns, also when the
    // persistent CTAs double-buffer their next tile with asynchronous copies (1023^2, one
    // instance: 43 us against 48-49 us); 32 x 32 tiles beat 32 x 8/16/40/64 rows
    const int grid = nitems;
#define HELM_RES(K, RR)                                                                        \
    (damp ? (mode ? launch_k(K<RR, 1, true>, dim3(grid), dim3(NTH), 0, s, insts, st, items, nitems, c)  \
                  : launch_k(K<RR, 0, true>, dim3(grid), dim3(NTH), 0, s, insts, st, items, nitems, c)) \
          : (mode ? launch_k(K<RR, 1, false>, dim3(grid), dim3(NTH), 0, s, insts, st, items, nitems, c) \
                  : launch_k(K<RR, 0, false>, dim3(grid), dim3(NTH), 0, s, insts, st, items, nitems, c)))
    if (D == 2 && prec == 0) HELM_RES(k_residual2d, double);
    else if (D == 2) HELM_RES(k_residual2d, float);
    else if (prec == 0) HELM_RES(k_residual3d, double);
    else HELM_RES(k_residual3d, float);
#undef HELM_RES
    return cudaGetLastError();
}

// tile width of the fused kernel: 32 (256-thread CTAs, four resident per SM, so CTAs in
// their smoothing phase and CTAs in their FP64 residual phase share each SM)
constexpr int UPX = 32;
// threads of the fused kernel (128 or 256; same results).  128 lets 7 CTAs share an SM, so
// a 1023^2 instance's 1024 tiles run in one wave, but measured slower (83.8 against
// 80.1 us per outer step): the CTAs' latency-bound phases want the 8 warps.
constexpr int UPRES_NT = 256;

int upres2d_tiles(int n) { return ((n + UPX - 1) / UPX) * ((n + UPY - 1) / UPY); }

cudaError_t launch_upres2d(const InstDesc* insts, InstState* st, const MgItem* items, int nitems, int n,
                           int nu2, int e2_mode, cudaStream_t s, int* ctrl, int nscan, int ninst,
                           int use_cond, unsigned long long cond_handle, int damp, int l1f)
{
    if (nitems <= 0) return cudaSuccess;
    const StepCtl c{ctrl, nscan, ninst, use_cond, cond_handle};
    const dim3 g(upres2d_tiles(n), nitems);
    const dim3 b(UPRES_NT);
#define HELM_UR(NU)                                                                                 \
    case NU:                                                                                        \
        if (l1f) {                                                                                  \
            if (damp) launch_k(k_upres2d<NU, true, UPRES_NT, true>, g, b, upres_bytes<NU, UPX, true>(), s, \
                               insts, st, items, e2_mode, c);                                       \
            else launch_k(k_upres2d<NU, false, UPRES_NT, true>, g, b, upres_bytes<NU, UPX, true>(), s,    \
                          insts, st, items, e2_mode, c);                                            \
        } else if (damp) launch_k(k_upres2d<NU, true, UPRES_NT, false>, g, b, upres_bytes<NU, UPX>(), s, \
                                  insts, st, items, e2_mode, c);                                    \
        else launch_k(k_upres2d<NU, false, UPRES_NT, false>, g, b, upres_bytes<NU, UPX>(), s, insts, st, \
                      items, e2_mode, c);                                                           \
        break;
    switch (nu2) {
        HELM_UR(0) HELM_UR(1) HELM_UR(2) HELM_UR(3) HELM_UR(4)
    default: return cudaErrorInvalidValue;
    }
#undef HELM_UR
    return cudaGetLastError();
}

template <int NU, bool L1F>
cudaError_t setup_upres_v()
{
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_upres2d<NU, false, UPRES_NT, L1F>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)upres_bytes<NU, UPX, L1F>())) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_upres2d<NU, true, UPRES_NT, L1F>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)upres_bytes<NU, UPX, L1F>())) != cudaSuccess) return e;
    if ((e = max_carveout(k_upres2d<NU, false, UPRES_NT, L1F>)) != cudaSuccess) return e;
    return max_carveout(k_upres2d<NU, true, UPRES_NT, L1F>);
}

template <int NU>
cudaError_t setup_upres()
{
    const cudaError_t e = setup_upres_v<NU, false>();
    return e != cudaSuccess ? e : setup_upres_v<NU, true>();
}

cudaError_t setup_outer()
{
    cudaError_t e;
#define HELM_CO(K)                                                                   \
    if ((e = max_carveout(K<float, 0, false>)) != cudaSuccess) return e;             \
    if ((e = max_carveout(K<float, 1, false>)) != cudaSuccess) return e;             \
    if ((e = max_carveout(K<double, 0, false>)) != cudaSuccess) return e;            \
    if ((e = max_carveout(K<double, 1, false>)) != cudaSuccess) return e;            \
    if ((e = max_carveout(K<float, 0, true>)) != cudaSuccess) return e;              \
    if ((e = max_carveout(K<float, 1, true>)) != cudaSuccess) return e;              \
    if ((e = max_carveout(K<double, 0, true>)) != cudaSuccess) return e;             \
    if ((e = max_carveout(K<double, 1, true>)) != cudaSuccess) return e;
    HELM_CO(k_residual2d)
    HELM_CO(k_residual3d)
#undef HELM_CO
    if ((e = setup_upres<0>()) != cudaSuccess) return e;
    if ((e = setup_upres<1>()) != cudaSuccess) return e;
    if ((e = setup_upres<2>()) != cudaSuccess) return e;
    if ((e = setup_upres<3>()) != cudaSuccess) return e;
    if ((e = setup_upres<4>()) != cudaSuccess) return e;
    return max_carveout(k_check);
}

cudaError_t launch_check(const InstState* st, int ninst, int* ctrl, int use_cond,
                         unsigned long long cond_handle, cudaStream_t s)
{
    launch_k(k_check, dim3(1), dim3(256), 0, s, st, ninst, ctrl, use_cond, cond_handle);
    return cudaGetLastError();
}

cudaError_t launch_fill_c128(void* p, long count, double re, double im, cudaStream_t s)
{
    launch_k(k_fill_c128, dim3(blocks_for(count)), dim3(256), 0, s, (double2*)p, count, re, im);
    return cudaGetLastError();
}

cudaError_t launch_max_re(int D, int n, const void* u, unsigned long long* out, cudaStream_t s)
{
    const long work = (D == 3) ? (long)n * n * n : (long)n * n;
    if (D == 2) launch_k(k_max_re<2>, dim3(blocks_for(work)), dim3(256), 0, s, (const double2*)u, n, out);
    else launch_k(k_max_re<3>, dim3(blocks_for(work)), dim3(256), 0, s, (const double2*)u, n, out);
    return cudaGetLastError();
}

#define HELM_DPR(K, ...)                                                                   \
    (D == 2 ? (prec == 0 ? launch_k(K<2, double>, __VA_ARGS__) : launch_k(K<2, float>, __VA_ARGS__)) \
            : (prec == 0 ? launch_k(K<3, double>, __VA_ARGS__) : launch_k(K<3, float>, __VA_ARGS__)))

cudaError_t launch_lev_fill(int D, int prec, const InstDesc* insts, int which, double value, cudaStream_t s)
{
    HELM_DPR(k_lev_fill, dim3(1216), dim3(256), 0, s, insts, which, value);
    return cudaGetLastError();
}

cudaError_t launch_lev_sumsq(int D, int prec, const InstDesc* insts, double* partial, double* out,
                             cudaStream_t s)
{
    HELM_DPR(k_lev_sumsq, dim3(PI_BLOCKS), dim3(256), 0, s, insts, partial);
    launch_k(k_sum_partials, dim3(1), dim3(32), 0, s, (const double*)partial, PI_BLOCKS, out);
    return cudaGetLastError();
}

cudaError_t launch_lev_scale(int D, int prec, const InstDesc* insts, double sc, cudaStream_t s)
{
    HELM_DPR(k_lev_scale, dim3(1216), dim3(256), 0, s, insts, sc);
    return cudaGetLastError();
}
#undef HELM_DPR

int power_iteration_blocks() { return PI_BLOCKS; }

cudaError_t launch_set_ring(int D, const InstDesc* insts, int inst, int n, cudaStream_t s)
{
    const long S = n + 2;
    const long work = (D == 3) ? S * S * S : S * S;
    if (D == 2) launch_k(k_set_ring<2>, dim3(blocks_for(work)), dim3(256), 0, s, insts, inst);
    else launch_k(k_set_ring<3>, dim3(blocks_for(work)), dim3(256), 0, s, insts, inst);
    return cudaGetLastError();
}

cudaError_t launch_set_ring_many(int D, const InstDesc* insts, const int* slots, int m, int n, cudaStream_t s)
{
    const long S = n + 2;
    const long work = (D == 3) ? S * S * S : S * S;
    for (int off = 0; off < m; off += 65535) {
        const int c = m - off < 65535 ? m - off : 65535;
        if (D == 2) launch_k(k_set_ring_many<2>, dim3(blocks_for(work), c), dim3(256), 0, s, insts, slots + off);
        else launch_k(k_set_ring_many<3>, dim3(blocks_for(work), c), dim3(256), 0, s, insts, slots + off);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_fill_res_many(ResItem* items, const int* slots, int m, int tx, int ty, int tz, cudaStream_t s)
{
    const int T = tx * ty * tz, total = m * T;
    if (total <= 0) return cudaSuccess;
    const int blocks = (total + 255) / 256 < 1024 ? (total + 255) / 256 : 1024;
    launch_k(k_fill_res_many, dim3(blocks), dim3(256), 0, s, items, slots, tx, ty, T, total);
    return cudaGetLastError();
}

cudaError_t launch_pack(int D, int prec, const InstDesc* insts, int inst, int n, const void* src,
                        int which, cudaStream_t s)
{
    const long work = (D == 3) ? (long)n * n * n : (long)n * n;
    const int nb = blocks_for(work);
    if (D == 2 && prec == 0) launch_k(k_pack<2, double>, dim3(nb), dim3(256), 0, s, insts, inst, src, which);
    else if (D == 2) launch_k(k_pack<2, float>, dim3(nb), dim3(256), 0, s, insts, inst, src, which);
    else if (prec == 0) launch_k(k_pack<3, double>, dim3(nb), dim3(256), 0, s, insts, inst, src, which);
    else launch_k(k_pack<3, float>, dim3(nb), dim3(256), 0, s, insts, inst, src, which);
    return cudaGetLastError();
}

cudaError_t launch_unpack(int D, int prec, const InstDesc* insts, int inst, int n, void* dst,
                          cudaStream_t s)
{
    const long work = (D == 3) ? (long)n * n * n : (long)n * n;
    const int nb = blocks_for(work);
    if (D == 2 && prec == 0) launch_k(k_unpack<2, double>, dim3(nb), dim3(256), 0, s, insts, inst, dst);
    else if (D == 2) launch_k(k_unpack<2, float>, dim3(nb), dim3(256), 0, s, insts, inst, dst);
    else if (prec == 0) launch_k(k_unpack<3, double>, dim3(nb), dim3(256), 0, s, insts, inst, dst);
    else launch_k(k_unpack<3, float>, dim3(nb), dim3(256), 0, s, insts, inst, dst);
    return cudaGetLastError();
}

}  // namespace helm
