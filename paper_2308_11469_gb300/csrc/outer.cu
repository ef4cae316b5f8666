// Outer (FP64) part of the Poisson iteration: the Helmholtz residual, the iterate
// update, the norms and the convergence test.
//
// One outer step of Section 2.2's iteration (alpha = k^2, p = 0) in residual form:
//   r_N = f - (Delta_h + k^2) u_N          (FP64, from the FP64 iterate)
//   Delta_h e_N = r_N, e_N = 0 on the wall (multigrid, inner precision)
//   u_{N+1} = u_N + e_N                    (FP64)
// i.e. Delta_h u_{N+1} = f - k^2 u_N; with exact solves e_N = v_N + i w_N.  The wall
// data g enters through the ring of u (the Dirichlet nodes of Section 2.4 that are moved
// to the right-hand side).
//
// k_residual (mode 1) fuses the update with the next residual: it forms
// u_{N+1} = u_N + e_N at a node and its 2D neighbours (e is zero on the ring), writes
// u_{N+1} to the other buffer of the ping-pong pair, and writes r_{N+1} (rounded to the
// inner precision) into the level-0 right-hand side; each tile leaves one partial
// sum of |r|^2 and one partial max |e| (fixed order => deterministic norms).
#include "launch.h"

namespace helm {
namespace {

constexpr int RES_BX = 32;
constexpr int RES_BY = 8;

template <int D> struct ResTile;
template <> struct ResTile<2> { static constexpr int RY = 4; };   // 32 x 32 nodes
template <> struct ResTile<3> { static constexpr int RY = 2; };   // 32 x 16 x 1 nodes

template <typename R>
__device__ __forceinline__ typename C2<R>::T to_inner(double2 v) {
    typename C2<R>::T o;
    o.x = (R)v.x;
    o.y = (R)v.y;
    return o;
}

template <int D, typename R, int MODE>
__global__ void __launch_bounds__(RES_BX * RES_BY)
k_residual(const InstDesc* __restrict__ insts, const InstState* __restrict__ st,
           const ResItem* __restrict__ items)
{
    typedef typename C2<R>::T c2;
    const ResItem item = items[blockIdx.x];
    const InstState s = st[item.inst];
    if (s.status != HELM_ST_ACTIVE) return;
    const InstDesc& I = insts[item.inst];
    const int n = I.n;
    const int S = n + 2;                      // tight padded row length of u / g
    const long SP = (long)S * S;
    const double2* __restrict__ uin = I.u[s.it & 1];
    double2* __restrict__ uout = I.u[(s.it + 1) & 1];
    const double2* __restrict__ f = I.f;
    const LevelDesc L0 = I.lev[0];
    const c2* __restrict__ e = (const c2*)L0.e;
    c2* __restrict__ rhs = (c2*)L0.rhs;
    const long P = L0.pitch;
    const long PL = (long)L0.pitch * L0.rows;
    const double ih2 = 1.0 / (I.h * I.h);
    const double k2 = I.k2;
    const double cdiag = k2 - 2.0 * D * ih2;

    const int x = item.tx * RES_BX + threadIdx.x + 1;
    const int z = (D == 3) ? item.tz + 1 : 0;
    double r2 = 0.0, emax = 0.0;
    constexpr int RY = ResTile<D>::RY;
#pragma unroll
    for (int k = 0; k < RY; ++k) {
        const int y = item.ty * (RES_BY * RY) + k * RES_BY + threadIdx.y + 1;
        if (x > n || y > n) continue;
        const long ou = ((D == 3) ? (long)z * SP : 0) + (long)y * S + x;
        const long oe = ((D == 3) ? (long)z * PL : 0) + (long)y * P + x;
        double2 c = uin[ou];
        double2 w = uin[ou - 1], ea = uin[ou + 1], so = uin[ou - S], no = uin[ou + S];
        double2 dn, up;
        if (D == 3) { dn = uin[ou - SP]; up = uin[ou + SP]; }
        if (MODE == 1) {
            const c2 e0 = e[oe];
            const c2 e1 = e[oe - 1], e2 = e[oe + 1], e3 = e[oe - P], e4 = e[oe + P];
            c.x += (double)e0.x;  c.y += (double)e0.y;
            w.x += (double)e1.x;  w.y += (double)e1.y;
            ea.x += (double)e2.x; ea.y += (double)e2.y;
            so.x += (double)e3.x; so.y += (double)e3.y;
            no.x += (double)e4.x; no.y += (double)e4.y;
            if (D == 3) {
                const c2 e5 = e[oe - PL], e6 = e[oe + PL];
                dn.x += (double)e5.x; dn.y += (double)e5.y;
                up.x += (double)e6.x; up.y += (double)e6.y;
            }
            uout[ou] = c;
            const double ex = (double)e0.x, ey = (double)e0.y;
            emax = fmax(emax, sqrt(ex * ex + ey * ey));
        }
        double sx = w.x + ea.x + so.x + no.x;
        double sy = w.y + ea.y + so.y + no.y;
        if (D == 3) {
            sx += dn.x + up.x;
            sy += dn.y + up.y;
        }
        const long of = (D == 3) ? ((long)(z - 1) * n + (y - 1)) * n + (x - 1)
                                 : (long)(y - 1) * n + (x - 1);
        const double2 fv = f[of];
        double2 r;
        r.x = fv.x - (sx * ih2 + cdiag * c.x);
        r.y = fv.y - (sy * ih2 + cdiag * c.y);
        rhs[oe] = to_inner<R>(r);
        r2 += r.x * r.x + r.y * r.y;
    }
    // deterministic block reduction: xor-shuffle within warps, then warps in order
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        r2 += __shfl_xor_sync(0xffffffffu, r2, o);
        emax = fmax(emax, __shfl_xor_sync(0xffffffffu, emax, o));
    }
    __shared__ double sr[RES_BY], sm[RES_BY];
    if (threadIdx.x == 0) {
        sr[threadIdx.y] = r2;
        sm[threadIdx.y] = emax;
    }
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        double a = 0.0, m = 0.0;
        for (int i = 0; i < RES_BY; ++i) {
            a += sr[i];
            m = fmax(m, sm[i]);
        }
        const int tid = (D == 3) ? (item.tz * I.res_ty + item.ty) * I.res_tx + item.tx
                                 : item.ty * I.res_tx + item.tx;
        I.part[tid] = a;
        I.part[I.nres_blocks + tid] = m;
    }
}

// One CTA; warp w handles instances w, w + 32, ...  Sums the partials in a fixed order,
// forms relres, applies the status rule, and (graph mode) sets the loop condition.
__global__ void __launch_bounds__(1024)
k_check(const InstDesc* __restrict__ insts, InstState* __restrict__ st, int ninst, int mode,
        int* __restrict__ ctrl, int use_cond, unsigned long long cond_handle)
{
    __shared__ int any_active;
    if (threadIdx.x == 0) any_active = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    for (int i = warp; i < ninst; i += nwarps) {
        InstState s = st[i];
        if (s.status != HELM_ST_ACTIVE) continue;
        const InstDesc& I = insts[i];
        double a = 0.0, m = 0.0;
        for (int b = lane; b < I.nres_blocks; b += 32) {
            a += I.part[b];
            m = fmax(m, I.part[I.nres_blocks + b]);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, o);
            m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
        }
        if (lane == 0) {
            const double norm = sqrt(a);
            double rel;
            int N;
            if (mode == 0) {
                N = 0;
                s.norm0 = norm;
                s.run = 0;
                rel = (norm == 0.0) ? 0.0 : 1.0;
            } else {
                s.it += 1;
                N = s.it;
                rel = norm / s.norm0;
                I.einf[N - 1] = m;
            }
            I.hist[N] = rel;
            int out = HELM_ST_ACTIVE;
            if (!isfinite(rel)) out = -4;                       // HELM_ENONFINITE
            else if (rel <= I.tol || (mode == 0 && norm == 0.0)) out = 0;   // CONVERGED
            else if (rel > 1e4) out = 2;                        // DIVERGED
            else {
                if (mode != 0) s.run = (rel >= s.prev) ? s.run + 1 : 0;
                if (N >= 20 && s.run >= 10) out = 2;            // DIVERGED
                else if (N >= I.max_outer) out = 1;             // MAXITER
            }
            s.prev = rel;
            s.status = out;
            st[i] = s;
            if (out == HELM_ST_ACTIVE) atomicOr(&any_active, 1);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int go = any_active;
        if (mode != 0) {
            const int done = ctrl[0] + 1;
            ctrl[0] = done;
            if (done >= ctrl[1]) go = 0;          // step budget of this launch
        }
        ctrl[2] = go;
        if (use_cond) cudaGraphSetConditional((cudaGraphConditionalHandle)cond_handle, go ? 1u : 0u);
    }
}

template <int D>
__global__ void k_set_ring(const InstDesc* __restrict__ insts, int inst)
{
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

template <int D, typename R>
__global__ void k_pack(const InstDesc* __restrict__ insts, int inst, const void* __restrict__ src,
                       int which)
{
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
        dst[((D == 3) ? ((long)z * L.rows + y) : (long)y) * L.pitch + x] = s[q];
    }
}

template <int D, typename R>
__global__ void k_unpack(const InstDesc* __restrict__ insts, int inst, void* __restrict__ dst)
{
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
        d[q] = src[((D == 3) ? ((long)z * L.rows + y) : (long)y) * L.pitch + x];
    }
}

inline int blocks_for(long work) {
    long b = (work + 255) / 256;
    if (b < 1) b = 1;
    if (b > 2432) b = 2432;
    return (int)b;
}

}  // namespace

cudaError_t launch_residual(int D, int prec, const InstDesc* insts, const InstState* st,
                            const ResItem* items, int nitems, int mode, cudaStream_t s)
{
    dim3 b(RES_BX, RES_BY);
    if (nitems <= 0) return cudaSuccess;
#define HELM_RES(DD, RR)                                                             \
    (mode ? (k_residual<DD, RR, 1><<<nitems, b, 0, s>>>(insts, st, items), 0)          \
          : (k_residual<DD, RR, 0><<<nitems, b, 0, s>>>(insts, st, items), 0))
    if (D == 2 && prec == 0) HELM_RES(2, double);
    else if (D == 2) HELM_RES(2, float);
    else if (prec == 0) HELM_RES(3, double);
    else HELM_RES(3, float);
#undef HELM_RES
    return cudaGetLastError();
}

cudaError_t launch_check(const InstDesc* insts, InstState* st, int ninst, int mode, int* ctrl,
                         int use_cond, unsigned long long cond_handle, cudaStream_t s)
{
    k_check<<<1, 1024, 0, s>>>(insts, st, ninst, mode, ctrl, use_cond, cond_handle);
    return cudaGetLastError();
}

cudaError_t launch_set_ring(int D, const InstDesc* insts, const InstState* st, int inst, int n,
                            cudaStream_t s)
{
    (void)st;
    const long S = n + 2;
    const long work = (D == 3) ? S * S * S : S * S;
    if (D == 2) k_set_ring<2><<<blocks_for(work), 256, 0, s>>>(insts, inst);
    else k_set_ring<3><<<blocks_for(work), 256, 0, s>>>(insts, inst);
    return cudaGetLastError();
}

cudaError_t launch_pack(int D, int prec, const InstDesc* insts, int inst, int n, const void* src,
                        int which, cudaStream_t s)
{
    const long work = (D == 3) ? (long)n * n * n : (long)n * n;
    const int nb = blocks_for(work);
    if (D == 2 && prec == 0) k_pack<2, double><<<nb, 256, 0, s>>>(insts, inst, src, which);
    else if (D == 2) k_pack<2, float><<<nb, 256, 0, s>>>(insts, inst, src, which);
    else if (prec == 0) k_pack<3, double><<<nb, 256, 0, s>>>(insts, inst, src, which);
    else k_pack<3, float><<<nb, 256, 0, s>>>(insts, inst, src, which);
    return cudaGetLastError();
}

cudaError_t launch_unpack(int D, int prec, const InstDesc* insts, int inst, int n, void* dst,
                          cudaStream_t s)
{
    const long work = (D == 3) ? (long)n * n * n : (long)n * n;
    const int nb = blocks_for(work);
    if (D == 2 && prec == 0) k_unpack<2, double><<<nb, 256, 0, s>>>(insts, inst, dst);
    else if (D == 2) k_unpack<2, float><<<nb, 256, 0, s>>>(insts, inst, dst);
    else if (prec == 0) k_unpack<3, double><<<nb, 256, 0, s>>>(insts, inst, dst);
    else k_unpack<3, float><<<nb, 256, 0, s>>>(insts, inst, dst);
    return cudaGetLastError();
}

}  // namespace helm
