// Coarse-level tail of the multigrid V-cycle: one CTA per instance runs every level
// with n <= 63 (2D) / n <= 15 (3D) in shared memory, down to the one-node exact solve
// e = -h^2 rhs / (2D), and back up.  Same operations, colours and weights as the
// global-memory levels (vcycle.cu / vcycle2d.cu): red-black Gauss-Seidel, residual,
// full weighting, multilinear prolongation.
//
// In complex64 the n = 31 level (2D) / n = 15 level (3D) is not cycled but solved exactly
// (a direct coarse-grid solver): the sine basis diagonalises Delta_h with zero walls, so
// e = (2/(n+1))^2 S ((S r S) / mu) S with S_ab = sin(pi a b / (n+1)) and
// mu_ab = -(4/h^2)(sin^2(pi a / (2(n+1))) + sin^2(pi b / (2(n+1)))).  The four 31 x 31
// products run on the FP32 pipes from shared memory.
//
// The level sizes are template parameters (n_top = 63, 31, ..., 1), so every index is
// compile-time arithmetic; lanes walk x, warps stride over rows.  Levels with n <= 7
// are run by warp 0 alone with warp-level barriers, the other warps wait at one block
// barrier.  Shared-memory layout: for each level, its iterate then its rhs, padded
// (n + 2)^D arrays with zero rings, each x-row stored with its even-x entries first and
// its odd-x entries after them, so that the lanes of a red-black half-sweep (one colour:
// x of one parity) and of the restriction read consecutive words (no bank conflicts).
#include <cmath>
#include <type_traits>

#include <cooperative_groups.h>

#include "launch.h"
#include "pdl.cuh"

namespace helm {
namespace {

namespace cg = cooperative_groups;

constexpr int TNT = 1024;

// Exact 2D solve of the n = 31 level (complex64)
constexpr int XN = 31;                 // level solved exactly
constexpr int XP = 32;                 // row pitch of the tables and of T2 (elements)
constexpr int XT = 34;                 // row pitch of the transposed intermediate (float2)
constexpr int XA = 4;                  // output rows per warp in the products
constexpr int XG = (XN + XA - 1) / XA; // warps of the products (8)
// scratch (floats): S[XN][XP], U[XN][XP], s[XP] (tables), Tt [XN][XT] float2,
// T2 [XN][XP] float2
constexpr int XTAB_FLOATS = 2 * XN * XP + XP;
constexpr int XSCR_FLOATS = XTAB_FLOATS + 2 * XN * XT + 2 * XN * XP;

// S_ab = sin(pi a b / 32), U_ab = 1 / (s_a + s_b) and s_a = sin^2(pi a / 64), written by
// setup_tail (host, double precision, rounded once)
__device__ float g_xtab[XTAB_FLOATS];

// Exact 3D solve of the n = 15 level (complex64): a sine transform along each axis, the
// diagonal scaling, and the transforms back.  Table: S[15][16] (S_ab = sin(pi a b / 16)),
// then s[16] (s_a = sin^2(pi a / 32)); scratch: two dense 15^3 complex buffers.
constexpr int YN = 15;
constexpr int YP = 16;
constexpr int YV = YN * YN * YN;
constexpr int YTAB_FLOATS = YN * YP + YP;
constexpr int YSCR_FLOATS = YTAB_FLOATS + 2 * 2 * YV;
__device__ float g_ytab[YTAB_FLOATS];

// Exact 2D solve of the n = 15 level in FP64 (the plain FP64 form): the same sine-basis
// formula with 15 x 15 products, a thread per output.  Table: S[15][16] (S_ab =
// sin(pi a b / 16)), then s[16] (s_a = sin^2(pi a / 32)); scratch: two 15 x 16 complex
// buffers.  (A 31 x 31 exact level in FP64 would cost ~60 us per cycle at one SM's FP64
// rate; at 15 it is ~7 us.)
constexpr int ZN = 15;
constexpr int ZP = 16;
constexpr int ZTAB_DOUBLES = ZN * ZP + ZP;
constexpr int ZSCR_DOUBLES = ZTAB_DOUBLES + 2 * 2 * ZN * ZP;
__device__ double g_ztab[ZTAB_DOUBLES];

template <int D, int N> struct Lv {
    static constexpr int S = N + 2;              // padded row length (odd)
    static constexpr int HE = (S + 1) / 2;       // even-x entries of a row, stored first
    static constexpr int SZ = (D == 3) ? S * S * S : S * S;
    static constexpr int NC = (N - 1) / 2;
};

// position of padded x within a row of a level with n = N
template <int N> __device__ __forceinline__ int ix(int x)
{
    return (x & 1) ? Lv<2, N>::HE + (x >> 1) : (x >> 1);
}

template <int D, int N> constexpr int tail_elems() {
    if constexpr (N <= 1) return 2 * Lv<D, 1>::SZ;
    else return 2 * Lv<D, N>::SZ + tail_elems<D, (N - 1) / 2>();
}

// the level each tail solves exactly (complex64: 2D 31, 3D 15; FP64: 2D 15, none in 3D)
template <int D, typename R> constexpr int exact_n()
{
    return std::is_same<R, float>::value ? (D == 2 ? XN : YN) : (D == 2 ? ZN : 0);
}

// does a tail with top size N0 contain its exactly solved level?
template <int D, typename R, int N0> constexpr bool tail_exact()
{
    return exact_n<D, R>() > 0 && N0 >= exact_n<D, R>();
}

template <int D, typename R, int N0> constexpr size_t tail_bytes()
{
    return (size_t)tail_elems<D, N0>() * sizeof(typename C2<R>::T) +
           (!tail_exact<D, R, N0>() ? 0
            : std::is_same<R, double>::value ? (size_t)ZSCR_DOUBLES * sizeof(double)
                                               : (size_t)(D == 2 ? XSCR_FLOATS : YSCR_FLOATS) * sizeof(float));
}

template <int NWARPS> __device__ __forceinline__ void tsync() {
    if constexpr (NWARPS == 1) __syncwarp();
    else __syncthreads();
}

template <typename T> __device__ __forceinline__ T cz() { T v; v.x = 0; v.y = 0; return v; }

template <int D, typename R, int N, int NWARPS>
__device__ __forceinline__ void t_sweep(typename C2<R>::T* E, const typename C2<R>::T* Rr, R h2,
                                        R dinv, int color)
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
        const int row = ((D == 3) ? (z * S + y) : y) * S;
        // x has the row's colour parity p; its west / east neighbours the other one
        constexpr int HE = Lv<D, N>::HE;
        const int p = xs & 1, m = row + (x >> 1);
        const int o = m + (p ? HE : 0);
        const c2 a = E[m + (p ? 0 : HE - 1)], b = E[m + (p ? 1 : HE)], c = E[o - S], d = E[o + S];
        R sx = a.x + b.x + c.x + d.x;
        R sy = a.y + b.y + c.y + d.y;
        if (D == 3) {
            const c2 f = E[o - S * S], g = E[o + S * S];
            sx += f.x + g.x;
            sy += f.y + g.y;
        }
        const c2 rr = Rr[o];
        c2 v;
        v.x = (sx - h2 * rr.x) * dinv;
        v.y = (sy - h2 * rr.y) * dinv;
        E[o] = v;
    }
}

// Full weighting of the residual rhs - Delta_h e; EZ: the iterate is known to be zero
// (no pre-smoothing from a zero guess), so the residual is rhs itself (the same values
// the general form yields with e = 0).
template <int D, typename R, int N, int NWARPS, bool EZ>
__device__ __forceinline__ void t_restrict(const typename C2<R>::T* E, const typename C2<R>::T* Rr,
                                           typename C2<R>::T* Rc, R h, R sig)
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
                    const int row = ((D == 3) ? ((2 * Z + dz) * S + 2 * Y + dy) : (2 * Y + dy)) * S;
                    const int x = 2 * X + dx;
                    const int o = row + ix<N>(x);
                    const c2 rr = Rr[o];
                    if constexpr (EZ) {
                        ax += w * rr.x;
                        ay += w * rr.y;
                    } else {
                        const c2 c = E[o], a = E[row + ix<N>(x - 1)], b = E[row + ix<N>(x + 1)];
                        const c2 u = E[o - S], d = E[o + S];
                        R sx = a.x + b.x + u.x + d.x;
                        R sy = a.y + b.y + u.y + d.y;
                        if (D == 3) {
                            const c2 f = E[o - S * S], g = E[o + S * S];
                            sx += f.x + g.x;
                            sy += f.y + g.y;
                        }
                        ax += w * ((rr.x - (sx - (R)(2 * D) * c.x) * ih2) + sig * c.x);
                        ay += w * ((rr.y - (sy - (R)(2 * D) * c.y) * ih2) + sig * c.y);
                    }
                }
            }
        }
        c2 v;
        v.x = ax * scale;
        v.y = ay * scale;
        Rc[((D == 3) ? (Z * SC + Y) : Y) * SC + ix<NC>(X)] = v;
    }
}

// e += multilinear interpolation of the coarse iterate.  Each row is walked by storage
// half: even x = 2q (coarse column q) then odd x = 2q + 1 (coarse columns q, q + 1), so
// lanes touch consecutive words.
template <int D, typename R, int N, int NWARPS>
__device__ __forceinline__ void t_prolong(typename C2<R>::T* E, const typename C2<R>::T* Ec)
{
    typedef typename C2<R>::T c2;
    constexpr int S = N + 2;
    constexpr int NC = (N - 1) / 2;
    constexpr int SC = NC + 2;
    constexpr int HE = Lv<D, N>::HE;
    constexpr int ROWS = (D == 3) ? N * N : N;
    const int lane = threadIdx.x & 31;
    const R w = (D == 3) ? (R)0.125 : (R)0.25;
    for (int r = threadIdx.x >> 5; r < ROWS; r += NWARPS) {
        const int y = r % N + 1;
        const int z = (D == 3) ? r / N + 1 : 0;
        const int row = ((D == 3) ? (z * S + y) : y) * S;
        const int y0 = y >> 1, y1 = (y + 1) >> 1;
        const int z0 = z >> 1, z1 = (z + 1) >> 1;
#pragma unroll
        for (int par = 0; par < 2; ++par) {
            const int q = lane + (par ? 0 : 1);
            if (2 * q + par > N) continue;
            const int c0 = ix<NC>(q), c1 = par ? ix<NC>(q + 1) : c0;
            R vx = 0, vy = 0;
#pragma unroll
            for (int iz = 0; iz < (D == 3 ? 2 : 1); ++iz)
#pragma unroll
                for (int iy = 0; iy < 2; ++iy) {
                    const int Z = iz ? z1 : z0, Y = iy ? y1 : y0;
                    const int crow = ((D == 3) ? (Z * SC + Y) : Y) * SC;
                    const c2 a = Ec[crow + c0], b = Ec[crow + c1];
                    vx += a.x;
                    vy += a.y;
                    vx += b.x;
                    vy += b.y;
                }
            const int o = row + (par ? HE : 0) + q;
            c2 v = E[o];
            v.x += w * vx;
            v.y += w * vy;
            E[o] = v;
        }
    }
}

// Clear the iterates of the levels the cycle will use (their rings must be zero and the
// coarse ones start from zero); the rhs arrays are written before they are read.
template <int D, typename R, int N>
__device__ __forceinline__ void t_clear(typename C2<R>::T* base)
{
    typedef typename C2<R>::T c2;
    for (int i = threadIdx.x; i < Lv<D, N>::SZ; i += TNT) base[i] = cz<c2>();
    constexpr bool exact_here = exact_n<D, R>() > 0 && N == exact_n<D, R>();
    if constexpr (N > 1 && !exact_here) t_clear<D, R, (N - 1) / 2>(base + 2 * Lv<D, N>::SZ);
}

// ---------------------------------------------------------------------------
// Exact 2D solve of the n = 31 level (complex64) in the sine basis
// ---------------------------------------------------------------------------
// element (y, x) (0-based interior indices) of a level array, or of a plain scratch
// matrix of pitch XP
template <bool LEVEL> __device__ __forceinline__ int x_at(int y, int x)
{
    if constexpr (LEVEL) return (y + 1) * (XN + 2) + ix<XN>(x + 1);
    else return y * XP + x;
}

// out_t[x][a] = sum_y S[a][y] in[y][x]: lanes over x, XA values of a per warp (S is
// symmetric, so S[a0..a0+3][y] is one float4 of row y)
template <bool LEVEL_IN>
__device__ __forceinline__ void x_cols(const float2* in, const float* Sm, float2* out_t)
{
    const int w = threadIdx.x >> 5, x = threadIdx.x & 31;
    if (w >= XG || x >= XN) return;
    const int a0 = XA * w;
    float2 acc[XA];
#pragma unroll
    for (int i = 0; i < XA; ++i) acc[i] = make_float2(0.f, 0.f);
#pragma unroll 8
    for (int y = 0; y < XN; ++y) {
        const float2 v = in[x_at<LEVEL_IN>(y, x)];
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

// out[a][b] = scale_ab * sum_x in_t[x][a] S[x][b] (scale_ab = c U_ab, or 1): lanes over
// b, XA values of a per warp.  With a shift (tau = sigma h^2 / 4 > 0) the scale is
// c / (s_a + s_b + tau) instead of c U_ab.
template <bool LEVEL_OUT>
__device__ __forceinline__ void x_rows(const float2* in_t, const float* Sm, const float* Um, float c,
                                       float tau, float2* out)
{
    const int w = threadIdx.x >> 5, b = threadIdx.x & 31;
    if (w >= XG || b >= XN) return;
    const int a0 = XA * w;
    float2 acc[XA];
#pragma unroll
    for (int i = 0; i < XA; ++i) acc[i] = make_float2(0.f, 0.f);
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
    for (int i = 0; i < XA; ++i) {
        const int a = a0 + i;
        if (a >= XN) break;
        float2 v = acc[i];
        if (Um) {
            const float* sv = Um + XN * XP;          // s_a follows the U table
            const float wv = (tau == 0.f) ? c * Um[a * XP + b] : c / (sv[a] + sv[b] + tau);
            v.x *= wv;
            v.y *= wv;
        }
        out[x_at<LEVEL_OUT>(a, b)] = v;
    }
}

// E (level array of n = 31) <- exact solution of (Delta_h - sigma) e = Rr with zero walls,
// h the level's spacing:  e = c S (U o (S r S)) S, c = -h^2 / (n+1)^2, with
// U_ab = 1 / (s_a + s_b + sigma h^2 / 4)
__device__ __forceinline__ void x_solve(float2* E, const float2* Rr, float* scr, float h, float sigma)
{
    const float* Sm = scr;
    const float* Um = scr + XN * XP;
    float2* Tt = reinterpret_cast<float2*>(scr + XTAB_FLOATS);
    float2* T2 = Tt + XN * XT;
    const float c = -(h * h) / (float)((XN + 1) * (XN + 1));
    const float tau = 0.25f * sigma * h * h;
    x_cols<true>(Rr, Sm, Tt);                  // S r          (transposed)
    __syncthreads();
    x_rows<false>(Tt, Sm, Um, c, tau, T2);     // c U o (S r S)
    __syncthreads();
    x_cols<false>(T2, Sm, Tt);                 // S (...)      (transposed)
    __syncthreads();
    x_rows<true>(Tt, Sm, nullptr, 1.f, 0.f, E);  // (S (...)) S
    __syncthreads();
}

// 3D: element (z, y, x) (0-based interior) of the n = 15 level array, or of a dense buffer
template <bool LEVEL> __device__ __forceinline__ int y_at(int z, int y, int x)
{
    constexpr int S = YN + 2;
    if constexpr (LEVEL) return ((z + 1) * S + (y + 1)) * S + ix<YN>(x + 1);
    else return (z * YN + y) * YN + x;
}

// One sine transform along `axis` (0 = x, 1 = y, 2 = z) of the 15^3 complex array:
// out[.., a, ..] = sum_j S[a][j] in[.., j, ..] (optionally scaled at the end); every thread
// forms whole outputs, the transformed index fastest for x, the x index fastest otherwise.
template <int AXIS, bool LEVEL_IN, bool LEVEL_OUT>
__device__ __forceinline__ void y_pass(const float2* in, float2* out, const float* Sm)
{
    for (int t = threadIdx.x; t < YV; t += TNT) {
        const int i0 = t % YN, i1 = (t / YN) % YN, i2 = t / (YN * YN);
        // (z, y, x) of the output; `a` is the transformed coordinate
        int z, y, x, a;
        if constexpr (AXIS == 0) { a = i0; y = i1; z = i2; x = 0; }
        else if constexpr (AXIS == 1) { x = i0; a = i1; z = i2; y = 0; }
        else { x = i0; y = i1; a = i2; z = 0; }
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll 5
        for (int j = 0; j < YN; ++j) {
            const float sv = Sm[j * YP + a];          // S is symmetric: lanes read along a row
            const float2 v = (AXIS == 0) ? in[y_at<LEVEL_IN>(z, y, j)]
                           : (AXIS == 1) ? in[y_at<LEVEL_IN>(z, j, x)] : in[y_at<LEVEL_IN>(j, y, x)];
            acc.x = fmaf(sv, v.x, acc.x);
            acc.y = fmaf(sv, v.y, acc.y);
        }
        if constexpr (AXIS == 0) out[y_at<LEVEL_OUT>(z, y, a)] = acc;
        else if constexpr (AXIS == 1) out[y_at<LEVEL_OUT>(z, a, x)] = acc;
        else out[y_at<LEVEL_OUT>(a, y, x)] = acc;
    }
}

// E (level array of n = 15, 3D) <- exact solution of (Delta_h - sigma) e = Rr, zero walls:
// e = c S S S ((S S S r) / (s_a + s_b + s_c + sigma h^2 / 4)), c = -2 h^2 / (n+1)^3
__device__ __forceinline__ void y_solve(float2* E, const float2* Rr, float* scr, float h, float sigma)
{
    const float* Sm = scr;
    const float* sv = scr + YN * YP;
    float2* T1 = reinterpret_cast<float2*>(scr + YTAB_FLOATS);
    float2* T2 = T1 + YV;
    const float c = -2.f * h * h / (float)((YN + 1) * (YN + 1) * (YN + 1));
    const float tau = 0.25f * sigma * h * h;
    y_pass<0, true, false>(Rr, T1, Sm);
    __syncthreads();
    y_pass<1, false, false>(T1, T2, Sm);
    __syncthreads();
    y_pass<2, false, false>(T2, T1, Sm);
    __syncthreads();
    for (int t = threadIdx.x; t < YV; t += TNT) {
        const int a = t % YN, b = (t / YN) % YN, cc = t / (YN * YN);
        const float w = c / (sv[a] + sv[b] + sv[cc] + tau);
        T1[t].x *= w;
        T1[t].y *= w;
    }
    __syncthreads();
    y_pass<2, false, false>(T1, T2, Sm);
    __syncthreads();
    y_pass<1, false, false>(T2, T1, Sm);
    __syncthreads();
    y_pass<0, false, true>(T1, E, Sm);
    __syncthreads();
}

// E (level array of n = 15, 2D, FP64) <- exact solution of (Delta_h - sigma) e = Rr with zero
// walls: e = c S (W o (S r S)) S, c = -h^2 / (n+1)^2, W_ab = 1 / (s_a + s_b + sigma h^2 / 4)
__device__ __forceinline__ void z_solve(double2* E, const double2* Rr, const double* scr, double h, double sigma)
{
    const double* Sm = scr;
    const double* sv = scr + ZN * ZP;
    double2* T1 = reinterpret_cast<double2*>(const_cast<double*>(scr) + ZTAB_DOUBLES);
    double2* T2 = T1 + ZN * ZP;
    const double c = -(h * h) / (double)((ZN + 1) * (ZN + 1));
    const double tau = 0.25 * sigma * h * h;
    const int t = threadIdx.x;
    const bool act = t < ZN * ZN;
    const int a = t / ZN, b = t % ZN;
    auto at = [](int y, int x) { return (y + 1) * (ZN + 2) + ix<ZN>(x + 1); };
    if (act) {                                   // T1[a][b] = sum_y S[a][y] r[y][b]
        double ax = 0.0, ay = 0.0;
        for (int y = 0; y < ZN; ++y) {
            const double s = Sm[a * ZP + y];
            const double2 v = Rr[at(y, b)];
            ax = fma(s, v.x, ax);
            ay = fma(s, v.y, ay);
        }
        T1[a * ZP + b] = make_double2(ax, ay);
    }
    __syncthreads();
    if (act) {                                   // T2[a][b] = c W_ab sum_x T1[a][x] S[x][b]
        double ax = 0.0, ay = 0.0;
        for (int x = 0; x < ZN; ++x) {
            const double s = Sm[x * ZP + b];
            const double2 v = T1[a * ZP + x];
            ax = fma(v.x, s, ax);
            ay = fma(v.y, s, ay);
        }
        const double w = c / (sv[a] + sv[b] + tau);
        T2[a * ZP + b] = make_double2(w * ax, w * ay);
    }
    __syncthreads();
    if (act) {                                   // T1[a][b] = sum_y S[a][y] T2[y][b]
        double ax = 0.0, ay = 0.0;
        for (int y = 0; y < ZN; ++y) {
            const double s = Sm[a * ZP + y];
            const double2 v = T2[y * ZP + b];
            ax = fma(s, v.x, ax);
            ay = fma(s, v.y, ay);
        }
        T1[a * ZP + b] = make_double2(ax, ay);
    }
    __syncthreads();
    if (act) {                                   // E[a][b] = sum_x T1[a][x] S[x][b]
        double ax = 0.0, ay = 0.0;
        for (int x = 0; x < ZN; ++x) {
            const double s = Sm[x * ZP + b];
            const double2 v = T1[a * ZP + x];
            ax = fma(v.x, s, ax);
            ay = fma(v.y, s, ay);
        }
        E[at(a, b)] = make_double2(ax, ay);
    }
    __syncthreads();
}

// One V(nu1, nu2)-cycle on the level of size N held at `base` (iterate, then rhs).
// ez: the iterate is zero on entry (a coarse level, or a top level started from zero).
// lv: this level's descriptor (its dinv); the next coarser level's follows it.
template <int D, typename R, int N, int NWARPS>
__device__ void t_vcycle(typename C2<R>::T* base, R h, R sig, const LevelDesc* lv, int nu1, int nu2,
                         float* xscr, bool ez)
{
    typedef typename C2<R>::T c2;
    c2* E = base;
    c2* Rr = base + Lv<D, N>::SZ;
    if constexpr (D == 2 && std::is_same<R, float>::value && N == XN && NWARPS == TNT / 32) {
        x_solve(E, Rr, xscr, (float)h, (float)sig);
        return;
    } else if constexpr (D == 3 && std::is_same<R, float>::value && N == YN && NWARPS == TNT / 32) {
        y_solve(E, Rr, xscr, (float)h, (float)sig);
        return;
    } else if constexpr (D == 2 && std::is_same<R, double>::value && N == ZN && NWARPS == TNT / 32) {
        z_solve(E, Rr, reinterpret_cast<const double*>(xscr), (double)h, (double)sig);
        return;
    } else if constexpr (N == 1) {
        if (threadIdx.x == 0) {
            constexpr int S = 3;
            constexpr int o = ((D == 3) ? (S + 1) : 1) * S + Lv<D, 1>::HE;  // the single node
            const c2 rr = Rr[o];
            const R c = -(h * h) * (R)lv->dinv;      // -h^2 / (2D + sigma h^2)
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
        const R dinv = (R)lv->dinv;                     // 1 / (2D + sigma h^2)
        for (int s = 0; s < nu1; ++s) {
            t_sweep<D, R, N, NWARPS>(E, Rr, h2, dinv, 0);
            tsync<NWARPS>();
            t_sweep<D, R, N, NWARPS>(E, Rr, h2, dinv, 1);
            tsync<NWARPS>();
        }
        if (ez && nu1 == 0) t_restrict<D, R, N, NWARPS, true>(E, Rr, Rc, h, sig);
        else t_restrict<D, R, N, NWARPS, false>(E, Rr, Rc, h, sig);
        tsync<NWARPS>();
        if constexpr (NWARPS > 1 && NC <= 7) {
            if (threadIdx.x < 32) t_vcycle<D, R, NC, 1>(Ec, h * (R)2, sig, lv + 1, nu1, nu2, xscr, true);
            __syncthreads();
        } else {
            t_vcycle<D, R, NC, NWARPS>(Ec, h * (R)2, sig, lv + 1, nu1, nu2, xscr, true);
        }
        t_prolong<D, R, N, NWARPS>(E, Ec);
        tsync<NWARPS>();
        for (int s = 0; s < nu2; ++s) {
            t_sweep<D, R, N, NWARPS>(E, Rr, h2, dinv, 0);
            tsync<NWARPS>();
            t_sweep<D, R, N, NWARPS>(E, Rr, h2, dinv, 1);
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
    const double sigma = insts[item.inst].sigma;
    pdl_wait();
    pdl_trigger();
    const InstState sv = st[item.inst];
    if (sv.status != HELM_ST_ACTIVE) return;
    if (L0.n != N0) return;                       // launched for another tail size
    constexpr int TOT = tail_elems<D, N0>();
    constexpr int S = N0 + 2;
    constexpr int ROWS = (D == 3) ? N0 * N0 : N0;
    const c2* __restrict__ gr = (const c2*)lev_rhs(L0, item.level, sv.it);
    const c2* __restrict__ ge = (const c2*)L0.e;
    // the starting iterate is read unless the top level is the exactly solved one (which
    // discards it)
    const bool le = load_e && item.level == 0 && !(tail_exact<D, R, N0>() && N0 == exact_n<D, R>());
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    c2* E = base;
    c2* Rr = base + Lv<D, N0>::SZ;
    // 2D: the top level's global loads go out first, their latency overlapping the
    // clearing of shared memory (3D: loaded after it, to bound the registers held)
    constexpr int RPW = (D == 2) ? (ROWS + 31) / 32 : 1;      // rows per warp
    constexpr int XJ = (N0 + 31) / 32;                         // 32-wide chunks of a row
    c2 vr[RPW][XJ], ve[RPW][XJ];
    if constexpr (D == 2) {
#pragma unroll
        for (int i = 0; i < RPW; ++i) {
            const int y = warp + 32 * i + 1;
#pragma unroll
            for (int j = 0; j < XJ; ++j) {
                const int x = lane + 32 * j + 1;
                if (y <= N0 && x <= N0) {
                    vr[i][j] = gr[(size_t)y * L0.pitch + x];
                    if (le) ve[i][j] = ge[(size_t)y * L0.pitch + x];
                }
            }
        }
    }
    float* xscr = nullptr;
    if constexpr (tail_exact<D, R, N0>()) {
        // sine tables of the exact level (host-computed)
        xscr = reinterpret_cast<float*>(base + TOT);
        if constexpr (std::is_same<R, double>::value) {
            constexpr int NT2 = ZTAB_DOUBLES / 2;
            const double2* tab = reinterpret_cast<const double2*>(g_ztab);
            for (int i = threadIdx.x; i < NT2; i += TNT) reinterpret_cast<double2*>(xscr)[i] = tab[i];
        } else {
            constexpr int NT4 = (D == 2 ? XTAB_FLOATS : YTAB_FLOATS) / 4;
            const float4* tab = reinterpret_cast<const float4*>(D == 2 ? g_xtab : g_ytab);
            for (int i = threadIdx.x; i < NT4; i += TNT) reinterpret_cast<float4*>(xscr)[i] = tab[i];
        }
    }
    t_clear<D, R, N0>(base);
    __syncthreads();
    if constexpr (D == 2) {
#pragma unroll
        for (int i = 0; i < RPW; ++i) {
            const int y = warp + 32 * i + 1;
#pragma unroll
            for (int j = 0; j < XJ; ++j) {
                const int x = lane + 32 * j + 1;
                if (y <= N0 && x <= N0) {
                    Rr[y * S + ix<N0>(x)] = vr[i][j];
                    if (le) E[y * S + ix<N0>(x)] = ve[i][j];
                }
            }
        }
    } else {
        for (int r = warp; r < ROWS; r += TNT / 32) {
            const int y = r % N0 + 1;
            const int z = r / N0 + 1;
            const size_t grow = ((size_t)z * L0.rows + y) * L0.pitch;
            const int srow = (z * S + y) * S;
#pragma unroll
            for (int j = 0; j < XJ; ++j) {
                const int x = lane + 32 * j + 1;
                if (x > N0) break;
                Rr[srow + ix<N0>(x)] = gr[grow + xslot<3>(x, L0.pitch)];
                if (le) E[srow + ix<N0>(x)] = ge[grow + xslot<3>(x, L0.pitch)];
            }
        }
    }
    __syncthreads();
    t_vcycle<D, R, N0, TNT / 32>(base, (R)L0.h, (R)sigma, &insts[item.inst].lev[item.level], nu1, nu2,
                                 xscr, !le);
    c2* __restrict__ go = (c2*)L0.e;
    for (int r = warp; r < ROWS; r += TNT / 32) {
        const int y = r % N0 + 1;
        const int z = (D == 3) ? r / N0 + 1 : 0;
        const size_t grow = ((D == 3) ? ((size_t)z * L0.rows + y) : (size_t)y) * L0.pitch;
        const int srow = ((D == 3) ? (z * S + y) : y) * S;
#pragma unroll
        for (int j = 0; j < XJ; ++j) {
            const int x = lane + 32 * j + 1;
            if (x > N0) break;
            go[grow + xslot<D>(x, L0.pitch)] = E[srow + ix<N0>(x)];
        }
    }
}

// ---------------------------------------------------------------------------
// Cluster tail (2D, complex64): levels 255, 127 and 63 in row bands over an 8-CTA
// thread-block cluster, the n = 31 level solved exactly (sine basis) in every CTA
// ---------------------------------------------------------------------------
// Used for cycles without pre-smoothing (nu1 = 0) whose level 255 is below the top, so
// every level the cluster runs starts from a zero iterate: the descent is the full
// weighting of the rhs, the ascent assigns the prolongation and smooths.  CTA k of the
// cluster owns rows 32k+1..32k+32 of level 255, 16k+1..16k+16 of level 127, 8k+1..8k+8 of
// level 63 and 4k+1..4k+4 of level 31.
//
//  * Descent: level 255's rhs rows 32k+1-(2 nu2-1) .. 32k+39 are staged from global memory;
//    each CTA restricts its own rows of every level plus the rows just below them that its
//    next restriction reads (levels 127: 16k+1..16k+19, 63: 8k+1..8k+9, 31: own), the extra
//    rows equal to their owners' values (same inputs, same operations).  One cluster barrier,
//    then every CTA copies from its neighbours' shared memory (distributed shared memory)
//    the other rhs rows its windows need; of level 31, all of them.
//  * Every CTA solves level 31 exactly from the same rhs: the same values in every CTA.
//  * Ascent: a CTA prolongs and smooths a window of rows around its band wide enough that
//    its final values are right where the next finer level reads them: a half-sweep
//    updates rows one closer to the band than the previous one (2 nu2 half-sweeps need 2
//    nu2 extra rows of the prolonged iterate and 2 nu2 - 1 of the rhs, per side), the
//    halo values being recomputed from the same inputs as the owner's.  No exchange is
//    needed on the way up; level 255's rhs window is staged again for its sweeps.
//
// Operations, colours and weights are those of the one-CTA tail and of the fused tile
// kernels (full weighting in the same order, the prolongation's four-corner sum, the
// half-sweep formula), so the cycle is the same.
constexpr int CT_CS = 8;                                   // CTAs per cluster
constexpr int CT_NA = 255, CT_NB = 127, CT_NC = 63;
constexpr int CT_SA = CT_NA + 2, CT_SB = CT_NB + 2, CT_SC = CT_NC + 2, CT_SX = XN + 2;

constexpr int fdiv2(int a) { return a >= 0 ? a / 2 : -((1 - a) / 2); }    // floor(a / 2)

// Row windows of CTA k (first row = band * k + OFF, ROWS rows) for nu2 = V.  F_l: rows
// of level l whose final values the next finer level's window reads.
template <int V> struct CtWin {
    // level 255: F = own rows; iterate F +- 2V, rhs F +- (2V - 1)
    static constexpr int EA_OFF = 1 - 2 * V, EA_ROWS = 32 + 4 * V;
    static constexpr int RA_OFF = 2 - 2 * V, RA_ROWS = (31 + 2 * V > 39 ? 31 + 2 * V : 39) - RA_OFF + 1;
    // level 127: F = [16k - V, 16k + 16 + V] (coarse rows of level 255's iterate window)
    static constexpr int FB_LO = -V, FB_HI = 16 + V;
    static constexpr int EB_OFF = FB_LO - 2 * V, EB_ROWS = FB_HI - FB_LO + 4 * V + 1;
    static constexpr int RB_OFF = FB_LO - (2 * V - 1);
    static constexpr int RB_ROWS = (FB_HI + 2 * V - 1 > 19 ? FB_HI + 2 * V - 1 : 19) - RB_OFF + 1;
    // level 63: F = coarse rows of level 127's iterate window
    static constexpr int FC_LO = fdiv2(EB_OFF), FC_HI = fdiv2(EB_OFF + EB_ROWS);
    static constexpr int EC_OFF = FC_LO - 2 * V, EC_ROWS = FC_HI - FC_LO + 4 * V + 1;
    static constexpr int RC_OFF = FC_LO - (2 * V - 1), RC_ROWS = FC_HI - FC_LO + 4 * V - 1;
    // shared memory (float2 units): level 255's iterate window, whose space holds levels 63
    // and 31 and the sine scratch until level 255 is prolonged; level 127's windows; level
    // 255's rhs window (staged once, read by the restriction and the last sweeps)
    static constexpr int O_EC = 0;
    static constexpr int O_RC = O_EC + EC_ROWS * CT_SC;
    static constexpr int O_EX = O_RC + RC_ROWS * CT_SC;
    static constexpr int O_RX = O_EX + CT_SX * CT_SX;
    static constexpr int O_SCR = (O_RX + CT_SX * CT_SX + 1) & ~1;        // 16-byte aligned
    static constexpr int A_WORDS = EA_ROWS * CT_SA;
    static constexpr int O_EB = (A_WORDS + 1) & ~1;
    static constexpr int O_RB = O_EB + EB_ROWS * CT_SB;
    static constexpr int O_RA = O_RB + RB_ROWS * CT_SB;
    static constexpr size_t BYTES = (size_t)(O_RA + RA_ROWS * CT_SA) * sizeof(float2);
    static_assert(O_SCR * 2 + XSCR_FLOATS <= 2 * A_WORDS, "levels 63 and 31 inside level 255's window");
    static_assert(BYTES <= 232448, "shared memory of one CTA");
};

// element (x, y) of a row window of a level with n = N whose first row is `lo`
template <int N> __device__ __forceinline__ int bw(int lo, int y, int x)
{
    return (y - lo) * (N + 2) + ix<N>(x);
}

// coarse rows [Ya, Yb] (within 1..NC) of the full weighting of the fine rhs window
template <int N>
__device__ __forceinline__ void ct_restrict(const float2* Rf, int flo, float2* Rc, int clo, int Ya, int Yb)
{
    constexpr int NC = (N - 1) / 2;
    const int lane = threadIdx.x & 31;
    Ya = max(Ya, 1);
    Yb = min(Yb, NC);
    for (int Y = Ya + (int)(threadIdx.x >> 5); Y <= Yb; Y += TNT / 32) {
        for (int X = lane + 1; X <= NC; X += 32) {
            float ax = 0.f, ay = 0.f;
#pragma unroll
            for (int dy = -1; dy <= 1; ++dy) {
                const float wy = (dy == 0) ? 2.f : 1.f;
#pragma unroll
                for (int dx = -1; dx <= 1; ++dx) {
                    const float w = wy * ((dx == 0) ? 2.f : 1.f);
                    const float2 rr = Rf[bw<N>(flo, 2 * Y + dy, 2 * X + dx)];
                    ax += w * rr.x;
                    ay += w * rr.y;
                }
            }
            float2 v;
            v.x = ax * (1.f / 16.f);
            v.y = ay * (1.f / 16.f);
            Rc[bw<NC>(clo, Y, X)] = v;
        }
    }
}

// fine rows [ya, yb] (within 1..N) of the window := multilinear interpolation of the coarse
// window (the fine iterate is zero: 0 + the interpolation, as the correction of a zero
// iterate rounds).  A lane forms the pair x = 2q + 1 (coarse columns q, q + 1) and x = 2q + 2
// (column q + 1 twice) from the same coarse words, summed in the order of the tile kernels:
// ((row y0 col 0 + row y0 col 1) + row y1 col 0) + row y1 col 1.
template <int N>
__device__ __forceinline__ void ct_prolong(float2* Ef, int flo, const float2* Ec, int clo, int ya, int yb)
{
    constexpr int NC = (N - 1) / 2;
    constexpr int S = N + 2, SC = NC + 2;
    constexpr int HE = Lv<2, N>::HE;
    const int lane = threadIdx.x & 31;
    ya = max(ya, 1);
    yb = min(yb, N);
    for (int y = ya + (int)(threadIdx.x >> 5); y <= yb; y += TNT / 32) {
        const int row = (y - flo) * S;
        const int r0 = ((y >> 1) - clo) * SC, r1 = (((y + 1) >> 1) - clo) * SC;
        for (int q = lane; q <= NC; q += 32) {
            const float2 a0 = Ec[r0 + ix<NC>(q)], a1 = Ec[r0 + ix<NC>(q + 1)];
            const float2 b0 = Ec[r1 + ix<NC>(q)], b1 = Ec[r1 + ix<NC>(q + 1)];
            float2 v;
            v.x = 0.f + 0.25f * (((a0.x + a1.x) + b0.x) + b1.x);
            v.y = 0.f + 0.25f * (((a0.y + a1.y) + b0.y) + b1.y);
            Ef[row + HE + q] = v;                            // x = 2q + 1
            if (q < NC) {                                    // x = 2q + 2
                v.x = 0.f + 0.25f * (((a1.x + a1.x) + b1.x) + b1.x);
                v.y = 0.f + 0.25f * (((a1.y + a1.y) + b1.y) + b1.y);
                Ef[row + q + 1] = v;
            }
        }
    }
}

// half-sweep of colour `color` on rows [ya, yb] (within 1..N) of the iterate window; the
// new values of rows [olo, ohi] also go to the level's global array `go` (row pitch P)
template <int N>
__device__ __forceinline__ void ct_sweep(float2* E, int elo, const float2* Rr, int rlo, int ya, int yb,
                                         float h2, float dinv, int color, float2* go = nullptr,
                                         int olo = 0, int ohi = -1, int P = 0, bool keep = true)
{
    constexpr int S = N + 2, HE = Lv<2, N>::HE;
    const int lane = threadIdx.x & 31;
    ya = max(ya, 1);
    yb = min(yb, N);
    for (int y = ya + (int)(threadIdx.x >> 5); y <= yb; y += TNT / 32) {
        const int xs = 1 + (((1 + y) & 1) ^ color);
        const int p = xs & 1;
        const int erow = (y - elo) * S, rrow = (y - rlo) * S;
        const bool out = go != nullptr && y >= olo && y <= ohi;
        for (int x = xs + 2 * lane; x <= N; x += 64) {
            const int m = x >> 1;
            const int oe = erow + m + (p ? HE : 0);
            const float2 a = E[erow + m + (p ? 0 : HE - 1)], b = E[erow + m + (p ? 1 : HE)];
            const float2 c = E[oe - S], d = E[oe + S];
            const float2 rr = Rr[rrow + m + (p ? HE : 0)];
            const float sx = a.x + b.x + c.x + d.x;
            const float sy = a.y + b.y + c.y + d.y;
            float2 v;
            v.x = (sx - h2 * rr.x) * dinv;
            v.y = (sy - h2 * rr.y) * dinv;
            if (keep) E[oe] = v;
            if (out) go[(size_t)y * P + x] = v;
        }
    }
}

// One rhs window to be completed from the CTAs that own its rows: rows [ya, yb] within 1..N
// and outside [lo_have, hi_have] (rows this CTA holds already); CTA o owns rows band*o + 1
// .. band*o + band and keeps them in its window starting at row wmul*o + off (wmul = band
// for a band window, 0 for a whole-level array).
struct CtPull {
    float2* W;
    int lo, ya, yb, lo_have, hi_have, band, wmul, off;
    __device__ int held() const { return max(0, min(hi_have, yb) - max(lo_have, ya) + 1); }
    __device__ int count() const { return max(0, yb - ya + 1) - held(); }
    // the i-th missing row
    __device__ int row(int i) const
    {
        const int y = ya + i;
        return (held() == 0 || y < max(lo_have, ya)) ? y : y + held();
    }
};

// copy the missing rows of three windows (levels 127, 63 and 31, S = 129, 65, 33 words):
// a warp per row, every remote word of a row loaded before any is stored
__device__ __forceinline__ void ct_pull3(cg::cluster_group& cl, CtPull p0, CtPull p1, CtPull p2)
{
    const int lane = threadIdx.x & 31;
    const int n0 = p0.count(), n1 = p1.count(), n2 = p2.count();
    for (int w = (int)(threadIdx.x >> 5); w < n0 + n1 + n2; w += TNT / 32) {
        CtPull p = p2;
        int i = w - n0 - n1, S = CT_SX;
        if (w < n0) {
            p = p0;
            i = w;
            S = CT_SB;
        } else if (w < n0 + n1) {
            p = p1;
            i = w - n0;
            S = CT_SC;
        }
        const int y = p.row(i);
        const int o = (y - 1) / p.band;
        const float2* src = cl.map_shared_rank(p.W, o) + (y - (p.wmul * o + p.off)) * S;
        float2* dst = p.W + (y - p.lo) * S;
        float2 v[5];
#pragma unroll
        for (int j = 0; j < 5; ++j)
            if (lane + 32 * j < S) v[j] = src[lane + 32 * j];
#pragma unroll
        for (int j = 0; j < 5; ++j)
            if (lane + 32 * j < S) dst[lane + 32 * j] = v[j];
    }
}

// cluster barrier halves: arrive releases this thread's shared-memory writes to the
// cluster, wait acquires those of every thread that arrived
__device__ __forceinline__ void ct_arrive() { asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory"); }
// (relaxed: this thread's loads from the other CTAs have completed, their values are used)
__device__ __forceinline__ void ct_arrive_relaxed() { asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory"); }
__device__ __forceinline__ void ct_wait() { asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory"); }

template <int V>
__global__ void __cluster_dims__(CT_CS, 1, 1) __launch_bounds__(TNT)
k_ctail(const InstDesc* __restrict__ insts, const InstState* __restrict__ st,
        const MgItem* __restrict__ items)
{
    typedef CtWin<V> W;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* base = reinterpret_cast<float2*>(smem_raw);
    cg::cluster_group cl = cg::this_cluster();
    const int k = (int)cl.block_rank();
    float2* EA = base;
    float2* EC = base + W::O_EC;
    float2* RC = base + W::O_RC;
    float2* EX = base + W::O_EX;
    float2* RX = base + W::O_RX;
    float* xscr = reinterpret_cast<float*>(base + W::O_SCR);
    float2* EB = base + W::O_EB;
    float2* RB = base + W::O_RB;
    float2* RA = base + W::O_RA;
    const int loEA = 32 * k + W::EA_OFF, loRA = 32 * k + W::RA_OFF;
    const int loEB = 16 * k + W::EB_OFF, loRB = 16 * k + W::RB_OFF;
    const int loEC = 8 * k + W::EC_OFF, loRC = 8 * k + W::RC_OFF;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // before the wait (nothing here depends on the predecessor): descriptors, the sine
    // tables, and the coarse iterate windows cleared (their rings and outer rows stay zero)
    const MgItem item = items[blockIdx.x / CT_CS];
    const LevelDesc LA = insts[item.inst].lev[item.level];
    const float dinvA = (float)LA.dinv;
    const float dinvB = (float)insts[item.inst].lev[item.level + 1].dinv;
    const float dinvC = (float)insts[item.inst].lev[item.level + 2].dinv;
    const float sig = (float)insts[item.inst].sigma;
    {
        constexpr int NT4 = XTAB_FLOATS / 4;
        const float4* tab = reinterpret_cast<const float4*>(g_xtab);
        for (int i = threadIdx.x; i < NT4; i += TNT) reinterpret_cast<float4*>(xscr)[i] = tab[i];
    }
    for (int i = threadIdx.x; i < W::EB_ROWS * CT_SB; i += TNT) EB[i] = make_float2(0.f, 0.f);
    for (int i = threadIdx.x; i < W::EC_ROWS * CT_SC; i += TNT) EC[i] = make_float2(0.f, 0.f);
    for (int i = threadIdx.x; i < CT_SX * CT_SX; i += TNT) EX[i] = make_float2(0.f, 0.f);
    pdl_wait();
    pdl_trigger();
    const InstState sv = st[item.inst];
    // every CTA of the cluster reads the same status and size: all leave together
    if (sv.status != HELM_ST_ACTIVE || LA.n != CT_NA) return;
    const float2* __restrict__ gr = (const float2*)lev_rhs(LA, item.level, sv.it);
    const int PA = LA.pitch;
    // level 255's rhs window, staged once: the descent reads its rows 32k+1 .. 32k+39, the
    // last sweeps rows 32k+1-(2 nu2-1) .. 32k+32+(2 nu2-1)
    for (int r = warp; r < W::RA_ROWS; r += TNT / 32) {
        const int y = loRA + r;
        if (y < 1 || y > CT_NA) continue;
        for (int x = lane + 1; x <= CT_NA; x += 32)
            cp_async_elem<8>(RA + bw<CT_NA>(loRA, y, x), gr + (size_t)y * PA + x, true);
    }
    cp_async_wait_all();
    __syncthreads();
    // descent: own rows of every level plus the rows below them the next restriction reads
    ct_restrict<CT_NA>(RA, loRA, RB, loRB, 16 * k + 1, 16 * k + 19);
    __syncthreads();
    ct_restrict<CT_NB>(RB, loRB, RC, loRC, 8 * k + 1, 8 * k + 9);
    __syncthreads();
    ct_restrict<CT_NC>(RC, loRC, RX, 0, 4 * k + 1, 4 * k + 4);
    ct_arrive();
    ct_wait();
    // the rhs rows of the windows held by the neighbours; level 31's whole rhs.  Then this
    // CTA has read the last of its neighbours' memory.
    {
        const CtPull pb{RB, loRB, max(loRB, 1), min(loRB + W::RB_ROWS - 1, CT_NB), 16 * k + 1,
                        min(16 * k + 19, CT_NB), 16, 16, W::RB_OFF};
        const CtPull pc{RC, loRC, max(loRC, 1), min(loRC + W::RC_ROWS - 1, CT_NC), 8 * k + 1,
                        min(8 * k + 9, CT_NC), 8, 8, W::RC_OFF};
        const CtPull px{RX, 0, 1, XN, 4 * k + 1, min(4 * k + 4, XN), 4, 0, 0};
        ct_pull3(cl, pb, pc, px);
    }
    __syncthreads();
    ct_arrive_relaxed();
    const float hA = (float)LA.h;
    x_solve(EX, RX, xscr, 8.f * hA, sig);
    // ascent: level 63 on its window
    ct_prolong<CT_NC>(EC, loEC, EX, 0, loEC, loEC + W::EC_ROWS - 1);
    __syncthreads();
    for (int s = 1; s <= 2 * V; ++s) {
        ct_sweep<CT_NC>(EC, loEC, RC, loRC, 8 * k + W::FC_LO - (2 * V - s), 8 * k + W::FC_HI + (2 * V - s),
                        (4.f * hA) * (4.f * hA), dinvC, (s - 1) & 1);
        __syncthreads();
    }
    ct_prolong<CT_NB>(EB, loEB, EC, loEC, loEB, loEB + W::EB_ROWS - 1);
    __syncthreads();
    for (int s = 1; s <= 2 * V; ++s) {
        ct_sweep<CT_NB>(EB, loEB, RB, loRB, 16 * k + W::FB_LO - (2 * V - s), 16 * k + W::FB_HI + (2 * V - s),
                        (2.f * hA) * (2.f * hA), dinvB, (s - 1) & 1);
        __syncthreads();
    }
    // the neighbours are done with this CTA's level-63 and level-31 rhs, which share level
    // 255's iterate window: zero its ring and outer rows, then assign its interior
    ct_wait();
    for (int r = warp; r < W::EA_ROWS; r += TNT / 32) {
        const int y = loEA + r;
        if (y >= 1 && y <= CT_NA) {
            if (lane < 2) EA[r * CT_SA + ix<CT_NA>(lane ? CT_NA + 1 : 0)] = make_float2(0.f, 0.f);
        } else {
            for (int x = lane; x < CT_SA; x += 32) EA[r * CT_SA + x] = make_float2(0.f, 0.f);
        }
    }
    ct_prolong<CT_NA>(EA, loEA, EB, loEB, loEA, loEA + W::EA_ROWS - 1);
    __syncthreads();
    // level 255's sweeps; the last half-sweep of each colour also writes the CTA's own rows
    // of the iterate to global memory (the very last one only there)
    float2* __restrict__ go = (float2*)LA.e;
    const int own_hi = min(32 * k + 32, CT_NA);
    for (int s = 1; s <= 2 * V; ++s) {
        const bool last = s >= 2 * V - 1;
        ct_sweep<CT_NA>(EA, loEA, RA, loRA, 32 * k + 1 - (2 * V - s), 32 * k + 32 + (2 * V - s), hA * hA, dinvA,
                        (s - 1) & 1, last ? go : nullptr, 32 * k + 1, own_hi, PA, s < 2 * V);
        if (s < 2 * V) __syncthreads();
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

template <int V>
cudaError_t ctail_attrs()
{
    cudaError_t e = cudaFuncSetAttribute(k_ctail<V>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)CtWin<V>::BYTES);
    if (e != cudaSuccess) return e;
    return max_carveout(k_ctail<V>);
}

// how many clusters of the kernel can be resident on this device at once (0: none)
template <int V>
int ctail_fits()
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(CT_CS);
    cfg.blockDim = dim3(TNT);
    cfg.dynamicSmemBytes = CtWin<V>::BYTES;
    int nc = 0;
    return cudaOccupancyMaxActiveClusters(&nc, k_ctail<V>, &cfg) == cudaSuccess ? nc : 0;
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
    const bool ex = tail_exact_n(D, prec) && n >= tail_exact_n(D, prec);
    return tot * elem + (!ex ? 0
                         : prec == 0 ? (size_t)ZSCR_DOUBLES * sizeof(double)
                                     : (size_t)(D == 2 ? XSCR_FLOATS : YSCR_FLOATS) * sizeof(float));
}

int tail_exact_n(int D, int prec) { return prec == 0 ? (D == 2 ? ZN : 0) : (D == 2 ? XN : YN); }

cudaError_t setup_tail(int D, int prec)
{
    if (D == 2 && prec != 0) {
        static float tab[XTAB_FLOATS];
        const double pi = 3.14159265358979323846;
        for (int i = 0; i < XN; ++i)
            for (int j = 0; j < XP; ++j) {
                const int a = i + 1, b = j + 1;
                const double sa = std::sin(pi * a / (2.0 * (XN + 1)));
                const double sb = std::sin(pi * b / (2.0 * (XN + 1)));
                const bool in = j < XN;
                tab[i * XP + j] = in ? (float)std::sin(pi * a * b / (XN + 1)) : 0.f;
                tab[XN * XP + i * XP + j] = in ? (float)(1.0 / (sa * sa + sb * sb)) : 0.f;
            }
        for (int i = 0; i < XP; ++i) {
            const double si = std::sin(pi * (i + 1) / (2.0 * (XN + 1)));
            tab[2 * XN * XP + i] = i < XN ? (float)(si * si) : 0.f;
        }
        const cudaError_t e = cudaMemcpyToSymbol(g_xtab, tab, sizeof tab);
        if (e != cudaSuccess) return e;
    }
    if (D == 2 && prec == 0) {
        static double tab[ZTAB_DOUBLES];
        const double pi = 3.14159265358979323846;
        for (int i = 0; i < ZN; ++i)
            for (int j = 0; j < ZP; ++j) tab[i * ZP + j] = j < ZN ? std::sin(pi * (i + 1) * (j + 1) / (ZN + 1)) : 0.0;
        for (int i = 0; i < ZP; ++i) {
            const double si = std::sin(pi * (i + 1) / (2.0 * (ZN + 1)));
            tab[ZN * ZP + i] = i < ZN ? si * si : 0.0;
        }
        const cudaError_t e = cudaMemcpyToSymbol(g_ztab, tab, sizeof tab);
        if (e != cudaSuccess) return e;
    }
    if (D == 3 && prec != 0) {
        static float tab[YTAB_FLOATS];
        const double pi = 3.14159265358979323846;
        for (int i = 0; i < YN; ++i)
            for (int j = 0; j < YP; ++j)
                tab[i * YP + j] = j < YN ? (float)std::sin(pi * (i + 1) * (j + 1) / (YN + 1)) : 0.f;
        for (int i = 0; i < YP; ++i) {
            const double si = std::sin(pi * (i + 1) / (2.0 * (YN + 1)));
            tab[YN * YP + i] = i < YN ? (float)(si * si) : 0.f;
        }
        const cudaError_t e = cudaMemcpyToSymbol(g_ytab, tab, sizeof tab);
        if (e != cudaSuccess) return e;
    }
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

int ctail_setup()
{
    static int ok = -1;
    if (ok < 0) {
        ok = 0;
        if (ctail_attrs<1>() == cudaSuccess && ctail_attrs<2>() == cudaSuccess) {
            const int a = ctail_fits<1>(), b = ctail_fits<2>();
            ok = a < b ? a : b;
        }
        cudaGetLastError();
    }
    return ok;
}

cudaError_t launch_ctail(const InstDesc* insts, const InstState* st, const MgItem* items, int nitems,
                         int nu2, cudaStream_t s)
{
    if (nu2 == 1)
        launch_k(k_ctail<1>, dim3(CT_CS * nitems), dim3(TNT), CtWin<1>::BYTES, s, insts, st, items);
    else if (nu2 == 2)
        launch_k(k_ctail<2>, dim3(CT_CS * nitems), dim3(TNT), CtWin<2>::BYTES, s, insts, st, items);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

}  // namespace helm
