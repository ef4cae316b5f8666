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

#include "launch.h"
#include "pdl.cuh"

namespace helm {
namespace {

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

}  // namespace helm
