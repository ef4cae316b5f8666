// Coarse-level tail of the multigrid V-cycle: one CTA per instance runs every level
// with n <= 63 (2D) / n <= 15 (3D) in shared memory, down to the one-node exact solve
// e = -h^2 rhs / (2D), and back up.  Same operations, colours and weights as the
// global-memory levels (vcycle.cu / vcycle2d.cu): red-black Gauss-Seidel, residual,
// full weighting, multilinear prolongation.
//
// In 2D complex64 the n = 31 level is not cycled but solved exactly (a direct
// coarse-grid solver): the sine basis diagonalises Delta_h with zero walls, so
// e = (2/(n+1))^2 S ((S r S) / mu) S with S_ab = sin(pi a b / (n+1)) and
// mu_ab = -(4/h^2)(sin^2(pi a / (2(n+1))) + sin^2(pi b / (2(n+1)))).  The four 31 x 31
// products run on the FP32 pipes from shared memory in ~1/4 of the barrier-bound time
// of the five-level cycle they replace.
//
// The level sizes are template parameters (n_top = 63, 31, ..., 1), so every index is
// compile-time arithmetic; lanes walk x, warps stride over rows.  Levels with n <= 7
// are run by warp 0 alone with warp-level barriers, the other warps wait at one block
// barrier.  Shared-memory layout: for each level, its iterate then its rhs, padded
// (n + 2)^D arrays with zero rings.
#include <type_traits>

#include "launch.h"
#include "pdl.cuh"

namespace helm {
namespace {

constexpr int TNT = 1024;

template <int D, int N> struct Lv {
    static constexpr int S = N + 2;
    static constexpr int SZ = (D == 3) ? S * S * S : S * S;
    static constexpr int NC = (N - 1) / 2;
};

template <int D, int N> constexpr int tail_elems() {
    if constexpr (N <= 1) return 2 * Lv<D, 1>::SZ;
    else return 2 * Lv<D, N>::SZ + tail_elems<D, (N - 1) / 2>();
}

// does a tail with top size N0 contain the exactly solved n = 31 level?
template <int D, typename R, int N0> constexpr bool tail_exact()
{
    return D == 2 && std::is_same<R, float>::value && N0 >= 31;
}

template <int D, typename R, int N0> constexpr size_t tail_bytes()
{
    return (size_t)tail_elems<D, N0>() * sizeof(typename C2<R>::T) +
           (tail_exact<D, R, N0>() ? (size_t)(2 * 31 * 32 + 2 * 31 * 34 + 2 * 31 * 32) * sizeof(float) : 0);
}

template <int NWARPS> __device__ __forceinline__ void tsync() {
    if constexpr (NWARPS == 1) __syncwarp();
    else __syncthreads();
}

template <typename T> __device__ __forceinline__ T cz() { T v; v.x = 0; v.y = 0; return v; }

template <int D, typename R, int N, int NWARPS>
__device__ __forceinline__ void t_sweep(typename C2<R>::T* E, const typename C2<R>::T* Rr, R h2,
                                        int color)
{
    typedef typename C2<R>::T c2;
    constexpr int S = N + 2;
    constexpr int ROWS = (D == 3) ? N * N : N;
    const int lane = threadIdx.x & 31;
    for (int r = threadIdx.x >> 5; r < ROWS; r += NWARPS) {
        const int y = r % N + 1;
        const int z = (D == 3) ? r / N + 1 : 0;
        const int xs = 1 + (((1 + y + z) & 1) ^ color);
        const int x = xs + 2 * lane;          // N <= 63: one pass of 32 lanes covers the row
        if (x > N) continue;
        const int o = ((D == 3) ? (z * S + y) : y) * S + x;
        const c2 a = E[o - 1], b = E[o + 1], c = E[o - S], d = E[o + S];
        R sx = a.x + b.x + c.x + d.x;
        R sy = a.y + b.y + c.y + d.y;
        if (D == 3) {
            const c2 f = E[o - S * S], g = E[o + S * S];
            sx += f.x + g.x;
            sy += f.y + g.y;
        }
        const c2 rr = Rr[o];
        c2 v;
        v.x = (sx - h2 * rr.x) * ((R)1 / (R)(2 * D));
        v.y = (sy - h2 * rr.y) * ((R)1 / (R)(2 * D));
        E[o] = v;
    }
}

template <int D, typename R, int N, int NWARPS>
__device__ __forceinline__ void t_restrict(const typename C2<R>::T* E, const typename C2<R>::T* Rr,
                                           typename C2<R>::T* Rc, R h)
{
    typedef typename C2<R>::T c2;
    constexpr int S = N + 2;
    constexpr int NC = (N - 1) / 2;
    constexpr int SC = NC + 2;
    constexpr int ROWS = (D == 3) ? NC * NC : NC;
    const R ih2 = (R)1 / (h * h);
    const R scale = (D == 3) ? (R)(1.0 / 64.0) : (R)(1.0 / 16.0);
    const int X = (threadIdx.x & 31) + 1;
    if (X > NC) return;
    for (int r = threadIdx.x >> 5; r < ROWS; r += NWARPS) {
        const int Y = r % NC + 1;
        const int Z = (D == 3) ? r / NC + 1 : 0;
        R ax = 0, ay = 0;
#pragma unroll
        for (int dz = (D == 3 ? -1 : 0); dz <= (D == 3 ? 1 : 0); ++dz) {
            const R wz = (D == 3) ? (dz == 0 ? (R)2 : (R)1) : (R)1;
#pragma unroll
            for (int dy = -1; dy <= 1; ++dy) {
                const R wy = (dy == 0) ? (R)2 : (R)1;
#pragma unroll
                for (int dx = -1; dx <= 1; ++dx) {
                    const R w = wz * wy * ((dx == 0) ? (R)2 : (R)1);
                    const int o = ((D == 3) ? ((2 * Z + dz) * S + 2 * Y + dy) : (2 * Y + dy)) * S + 2 * X + dx;
                    const c2 c = E[o], a = E[o - 1], b = E[o + 1], u = E[o - S], d = E[o + S];
                    R sx = a.x + b.x + u.x + d.x;
                    R sy = a.y + b.y + u.y + d.y;
                    if (D == 3) {
                        const c2 f = E[o - S * S], g = E[o + S * S];
                        sx += f.x + g.x;
                        sy += f.y + g.y;
                    }
                    const c2 rr = Rr[o];
                    ax += w * (rr.x - (sx - (R)(2 * D) * c.x) * ih2);
                    ay += w * (rr.y - (sy - (R)(2 * D) * c.y) * ih2);
                }
            }
        }
        c2 v;
        v.x = ax * scale;
        v.y = ay * scale;
        Rc[((D == 3) ? (Z * SC + Y) : Y) * SC + X] = v;
    }
}

template <int D, typename R, int N, int NWARPS>
__device__ __forceinline__ void t_prolong(typename C2<R>::T* E, const typename C2<R>::T* Ec)
{
    typedef typename C2<R>::T c2;
    constexpr int S = N + 2;
    constexpr int NC = (N - 1) / 2;
    constexpr int SC = NC + 2;
    constexpr int ROWS = (D == 3) ? N * N : N;
    const int lane = threadIdx.x & 31;
    for (int r = threadIdx.x >> 5; r < ROWS; r += NWARPS) {
        const int y = r % N + 1;
        const int z = (D == 3) ? r / N + 1 : 0;
        const int y0 = y >> 1, y1 = (y + 1) >> 1;
        const int z0 = z >> 1, z1 = (z + 1) >> 1;
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int x = lane + 32 * j + 1;
            if (x > N) break;
            const int x0 = x >> 1, x1 = (x + 1) >> 1;
            R vx = 0, vy = 0;
#pragma unroll
            for (int iz = 0; iz < (D == 3 ? 2 : 1); ++iz)
#pragma unroll
                for (int iy = 0; iy < 2; ++iy)
#pragma unroll
                    for (int ix = 0; ix < 2; ++ix) {
                        const int Z = iz ? z1 : z0, Y = iy ? y1 : y0, XX = ix ? x1 : x0;
                        const c2 c = Ec[((D == 3) ? (Z * SC + Y) : Y) * SC + XX];
                        vx += c.x;
                        vy += c.y;
                    }
            const R w = (D == 3) ? (R)0.125 : (R)0.25;
            const int o = ((D == 3) ? (z * S + y) : y) * S + x;
            c2 v = E[o];
            v.x += w * vx;
            v.y += w * vy;
            E[o] = v;
        }
    }
}

// ---------------------------------------------------------------------------
// Exact 2D solve on the n = 31 level (complex64) in the sine basis
// ---------------------------------------------------------------------------
constexpr int XN = 31;                 // level solved exactly (2D complex64)
constexpr int XP = 32;                 // row pitch of the tables and of T2 (elements)
constexpr int XT = 34;                 // row pitch of the transposed intermediates (float2)
constexpr int XGROUPS = (XN + 3) / 4;  // warps of the products, 4 output rows each

// scratch (floats): S[XN][XP], W[XN][XP], Tt[XN][XT] float2, T2[XN][XP] float2
constexpr int XSCR_FLOATS = 2 * XN * XP + 2 * XN * XT + 2 * XN * XP;

// out_t[x][a] = sum_y S[a][y] in[y][x]  (lanes over x, 4 values of a per warp; S is
// symmetric, so S[a..a+3][y] is one float4 of row y)
__device__ __forceinline__ void x_cols(const float2* in, int in_pitch, int in_off,
                                       const float* Sm, float2* out_t)
{
    const int w = threadIdx.x >> 5, x = threadIdx.x & 31;
    if (w >= XGROUPS || x >= XN) return;
    const int a0 = 4 * w;
    float2 acc[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) acc[i] = make_float2(0.f, 0.f);
#pragma unroll 8
    for (int y = 0; y < XN; ++y) {
        const float2 v = in[in_off + y * in_pitch + x];
        const float4 s4 = *reinterpret_cast<const float4*>(Sm + y * XP + a0);
        acc[0].x = fmaf(s4.x, v.x, acc[0].x); acc[0].y = fmaf(s4.x, v.y, acc[0].y);
        acc[1].x = fmaf(s4.y, v.x, acc[1].x); acc[1].y = fmaf(s4.y, v.y, acc[1].y);
        acc[2].x = fmaf(s4.z, v.x, acc[2].x); acc[2].y = fmaf(s4.z, v.y, acc[2].y);
        acc[3].x = fmaf(s4.w, v.x, acc[3].x); acc[3].y = fmaf(s4.w, v.y, acc[3].y);
    }
    float4* o = reinterpret_cast<float4*>(out_t + x * XT + a0);
    o[0] = make_float4(acc[0].x, acc[0].y, acc[1].x, acc[1].y);
    o[1] = make_float4(acc[2].x, acc[2].y, acc[3].x, acc[3].y);
}

// out[a][b] = W[a][b] * sum_x in_t[x][a] S[x][b]  (lanes over b, 4 values of a per warp)
__device__ __forceinline__ void x_rows(const float2* in_t, const float* Sm, const float* Wm,
                                       float2* out, int out_pitch, int out_off)
{
    const int w = threadIdx.x >> 5, b = threadIdx.x & 31;
    if (w >= XGROUPS || b >= XN) return;
    const int a0 = 4 * w;
    float2 acc[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) acc[i] = make_float2(0.f, 0.f);
#pragma unroll 8
    for (int x = 0; x < XN; ++x) {
        const float s = Sm[x * XP + b];
        const float4* t = reinterpret_cast<const float4*>(in_t + x * XT + a0);
        const float4 t01 = t[0], t23 = t[1];
        acc[0].x = fmaf(t01.x, s, acc[0].x); acc[0].y = fmaf(t01.y, s, acc[0].y);
        acc[1].x = fmaf(t01.z, s, acc[1].x); acc[1].y = fmaf(t01.w, s, acc[1].y);
        acc[2].x = fmaf(t23.x, s, acc[2].x); acc[2].y = fmaf(t23.y, s, acc[2].y);
        acc[3].x = fmaf(t23.z, s, acc[3].x); acc[3].y = fmaf(t23.w, s, acc[3].y);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int a = a0 + i;
        if (a >= XN) break;
        float2 v = acc[i];
        if (Wm) {
            const float wv = Wm[a * XP + b];
            v.x *= wv;
            v.y *= wv;
        }
        out[out_off + a * out_pitch + b] = v;
    }
}

// Tables of the sine basis for the n = 31 level of spacing h: S and the scaled inverse
// eigenvalues W_ab = (2/(n+1))^2 / mu_ab = -h^2 / ((n+1)^2 (s_a + s_b)),
// s_a = sin^2(pi a / (2(n+1))).  Written once per CTA before the cycle starts.
__device__ __forceinline__ void x_tables(float* scr, float h)
{
    float* Sm = scr;
    float* Wm = scr + XN * XP;
    const float c = -(h * h) / (float)((XN + 1) * (XN + 1));
    for (int q = threadIdx.x; q < XN * XP; q += blockDim.x) {
        const int i = q / XP, j = q % XP;
        if (j >= XN) { Sm[q] = 0.f; Wm[q] = 0.f; continue; }
        const int a = i + 1, b = j + 1;
        Sm[q] = sinpif((float)((a * b) % (2 * (XN + 1))) / (float)(XN + 1));
        const float sa = sinpif((float)a / (float)(2 * (XN + 1)));
        const float sb = sinpif((float)b / (float)(2 * (XN + 1)));
        Wm[q] = c / (sa * sa + sb * sb);
    }
}

// E (padded (n+2)^2, pitch n+2) <- exact solution of Delta_h e = Rr with zero walls
__device__ __forceinline__ void x_solve(float2* E, const float2* Rr, float* scr)
{
    const float* Sm = scr;
    const float* Wm = scr + XN * XP;
    float2* Tt = reinterpret_cast<float2*>(scr + 2 * XN * XP);
    float2* T2 = Tt + XN * XT;
    constexpr int SP = XN + 2;
    x_cols(Rr, SP, SP + 1, Sm, Tt);            // S r          (transposed)
    __syncthreads();
    x_rows(Tt, Sm, Wm, T2, XP, 0);             // W (S r S)
    __syncthreads();
    x_cols(T2, XP, 0, Sm, Tt);                 // S (...)      (transposed)
    __syncthreads();
    x_rows(Tt, Sm, nullptr, E, SP, SP + 1);    // (S (...)) S
    __syncthreads();
}

template <int D, typename R, int N, int NWARPS>
__device__ void t_vcycle(typename C2<R>::T* base, R h, int nu1, int nu2, float* xscr)
{
    typedef typename C2<R>::T c2;
    c2* E = base;
    c2* Rr = base + Lv<D, N>::SZ;
    if constexpr (D == 2 && std::is_same<R, float>::value && N == XN && NWARPS == TNT / 32) {
        x_solve(E, Rr, xscr);
        return;
    } else if constexpr (N == 1) {
        if (threadIdx.x == 0) {
            constexpr int o = (D == 3) ? 13 : 4;   // the single interior node
            const c2 rr = Rr[o];
            const R c = -(h * h) / (R)(2 * D);
            c2 v;
            v.x = c * rr.x;
            v.y = c * rr.y;
            E[o] = v;
        }
        tsync<NWARPS>();
    } else {
        constexpr int NC = (N - 1) / 2;
        c2* Ec = base + 2 * Lv<D, N>::SZ;
        c2* Rc = Ec + Lv<D, NC>::SZ;
        const R h2 = h * h;
        for (int s = 0; s < nu1; ++s) {
            t_sweep<D, R, N, NWARPS>(E, Rr, h2, 0);
            tsync<NWARPS>();
            t_sweep<D, R, N, NWARPS>(E, Rr, h2, 1);
            tsync<NWARPS>();
        }
        t_restrict<D, R, N, NWARPS>(E, Rr, Rc, h);
        tsync<NWARPS>();
        if constexpr (NWARPS > 1 && NC <= 7) {
            if (threadIdx.x < 32) t_vcycle<D, R, NC, 1>(Ec, h * (R)2, nu1, nu2, xscr);
            __syncthreads();
        } else {
            t_vcycle<D, R, NC, NWARPS>(Ec, h * (R)2, nu1, nu2, xscr);
        }
        t_prolong<D, R, N, NWARPS>(E, Ec);
        tsync<NWARPS>();
        for (int s = 0; s < nu2; ++s) {
            t_sweep<D, R, N, NWARPS>(E, Rr, h2, 0);
            tsync<NWARPS>();
            t_sweep<D, R, N, NWARPS>(E, Rr, h2, 1);
            tsync<NWARPS>();
        }
    }
}

template <int D, typename R, int N0>
__global__ void __launch_bounds__(TNT)
k_tail(const InstDesc* __restrict__ insts, const InstState* __restrict__ st,
       const MgItem* __restrict__ items, int nu1, int nu2, int load_e)
{
    typedef typename C2<R>::T c2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    c2* base = reinterpret_cast<c2*>(smem_raw);
    const MgItem item = items[blockIdx.x];
    const LevelDesc L0 = insts[item.inst].lev[item.level];   // host-written: read before the wait
    pdl_wait();
    pdl_trigger();
    if (st[item.inst].status != HELM_ST_ACTIVE) return;
    if (L0.n != N0) return;                       // launched for another tail size
    constexpr int TOT = tail_elems<D, N0>();
    for (int i = threadIdx.x; i < TOT; i += TNT) base[i] = cz<c2>();
    float* xscr = nullptr;
    if constexpr (tail_exact<D, R, N0>()) {
        xscr = reinterpret_cast<float*>(base + TOT);
        // the level spacing of n = 31 under the top level's h
        x_tables(xscr, (float)L0.h * (float)((N0 + 1) / (XN + 1)));
    }
    __syncthreads();
    constexpr int S = N0 + 2;
    constexpr int ROWS = (D == 3) ? N0 * N0 : N0;
    const c2* __restrict__ gr = (const c2*)L0.rhs;
    const c2* __restrict__ ge = (const c2*)L0.e;
    const bool le = load_e && item.level == 0;
    const int lane = threadIdx.x & 31;
    c2* E = base;
    c2* Rr = base + Lv<D, N0>::SZ;
    for (int r = threadIdx.x >> 5; r < ROWS; r += TNT / 32) {
        const int y = r % N0 + 1;
        const int z = (D == 3) ? r / N0 + 1 : 0;
        const size_t grow = ((D == 3) ? ((size_t)z * L0.rows + y) : (size_t)y) * L0.pitch;
        const int srow = ((D == 3) ? (z * S + y) : y) * S;
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int x = lane + 32 * j + 1;
            if (x > N0) break;
            Rr[srow + x] = gr[grow + x];
            if (le) E[srow + x] = ge[grow + x];
        }
    }
    __syncthreads();
    t_vcycle<D, R, N0, TNT / 32>(base, (R)L0.h, nu1, nu2, xscr);
    c2* __restrict__ go = (c2*)L0.e;
    for (int r = threadIdx.x >> 5; r < ROWS; r += TNT / 32) {
        const int y = r % N0 + 1;
        const int z = (D == 3) ? r / N0 + 1 : 0;
        const size_t grow = ((D == 3) ? ((size_t)z * L0.rows + y) : (size_t)y) * L0.pitch;
        const int srow = ((D == 3) ? (z * S + y) : y) * S;
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int x = lane + 32 * j + 1;
            if (x > N0) break;
            go[grow + x] = E[srow + x];
        }
    }
}

template <int D, typename R, int N0>
cudaError_t tl(const InstDesc* insts, const InstState* st, const MgItem* items, int nitems,
               int nu1, int nu2, int load_e, cudaStream_t s)
{
    const size_t sm = tail_bytes<D, R, N0>();
    launch_k(k_tail<D, R, N0>, dim3(nitems), dim3(TNT), sm, s, insts, st, items, nu1, nu2, load_e);
    return cudaGetLastError();
}

template <int D, typename R, int N0>
cudaError_t ta()
{
    const size_t sm = tail_bytes<D, R, N0>();
    const cudaError_t e = cudaFuncSetAttribute(k_tail<D, R, N0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    return max_carveout(k_tail<D, R, N0>);
}

template <int D, typename R>
cudaError_t tail_dispatch(int n0, const InstDesc* insts, const InstState* st, const MgItem* items,
                          int nitems, int nu1, int nu2, int load_e, cudaStream_t s)
{
    switch (n0) {
    case 1: return tl<D, R, 1>(insts, st, items, nitems, nu1, nu2, load_e, s);
    case 3: return tl<D, R, 3>(insts, st, items, nitems, nu1, nu2, load_e, s);
    case 7: return tl<D, R, 7>(insts, st, items, nitems, nu1, nu2, load_e, s);
    case 15: return tl<D, R, 15>(insts, st, items, nitems, nu1, nu2, load_e, s);
    case 31: if (D == 2) return tl<2, R, 31>(insts, st, items, nitems, nu1, nu2, load_e, s); break;
    case 63: if (D == 2) return tl<2, R, 63>(insts, st, items, nitems, nu1, nu2, load_e, s); break;
    default: break;
    }
    return cudaErrorInvalidValue;
}

template <int D, typename R>
cudaError_t tail_attrs()
{
    cudaError_t e;
    if ((e = ta<D, R, 1>()) != cudaSuccess) return e;
    if ((e = ta<D, R, 3>()) != cudaSuccess) return e;
    if ((e = ta<D, R, 7>()) != cudaSuccess) return e;
    if ((e = ta<D, R, 15>()) != cudaSuccess) return e;
    if constexpr (D == 2) {
        if ((e = ta<2, R, 31>()) != cudaSuccess) return e;
        if ((e = ta<2, R, 63>()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace

size_t tail_smem_bytes(int D, int prec, int n)
{
    size_t elem = prec == 0 ? 16 : 8;
    size_t tot = 0;
    for (int m = n; m >= 1; m = (m - 1) >> 1) {
        size_t s = (size_t)(m + 2);
        tot += 2 * ((D == 3) ? s * s * s : s * s);
    }
    return tot * elem + (size_t)(tail_exact_n(D, prec) && n >= tail_exact_n(D, prec) ? XSCR_FLOATS * sizeof(float) : 0);
}

int tail_exact_n(int D, int prec) { return (D == 2 && prec != 0) ? XN : 0; }

cudaError_t setup_tail(int D, int prec)
{
    if (D == 2) return prec == 0 ? tail_attrs<2, double>() : tail_attrs<2, float>();
    return prec == 0 ? tail_attrs<3, double>() : tail_attrs<3, float>();
}

cudaError_t launch_tail(int D, int prec, int n0, const InstDesc* insts, const InstState* st,
                        const MgItem* items, int nitems, int nu1, int nu2, int load_e, cudaStream_t s)
{
    if (D == 2)
        return prec == 0 ? tail_dispatch<2, double>(n0, insts, st, items, nitems, nu1, nu2, load_e, s)
                         : tail_dispatch<2, float>(n0, insts, st, items, nitems, nu1, nu2, load_e, s);
    return prec == 0 ? tail_dispatch<3, double>(n0, insts, st, items, nitems, nu1, nu2, load_e, s)
                     : tail_dispatch<3, float>(n0, insts, st, items, nitems, nu1, nu2, load_e, s);
}

}  // namespace helm
