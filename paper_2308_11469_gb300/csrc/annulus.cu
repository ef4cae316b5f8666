// The annular problem (Section 2.3 and the FD discussion of Section 2.4): a square with a
// square hole, Dirichlet data on the hole, a Robin condition du/dn - i k u = q on the
// outer edge.
//
// Grid: [-side/2, side/2]^2 with N intervals per axis (N a power of two), h = side / N,
// node (i, j) at (-side/2 + i h, -side/2 + j h), stored at i (N + 1) + j.  Node types:
// HOLE (|x|, |y| <= hole: Dirichlet, value g), EDGE (i or j in {0, N}: the row is the
// outward normal derivative, the one-sided difference towards the inward neighbour,
// averaged over the two normals at a corner), PDE (5-point Delta_h).
//
// Outer iteration (FP64, Section 2.3 in residual form, sigma = alpha - k^2 >= 0):
//   r_N = b - B U_N,  A_sigma e_N = r_N,  U_{N+1} = U_N + e_N,
// B: PDE rows Delta_h + k^2, EDGE rows d/dn - i k;  A_sigma: PDE rows Delta_h - sigma,
// EDGE rows d/dn.  With exact inner solves the partial sums are those of the paper's
// v_n + i w_n (Neumann data -k w_{n-1}, +k v_{n-1} on the outer edge).
//
// Inner solve: multigrid V-cycles in the inner precision on rediscretised levels N, N/2,
// ..., 8 (node types by the same rule at each level; the coarsest solved exactly through a
// host-computed inverse).  Red-black Gauss-Seidel solves each row by its own equation;
// the residual is restricted by full weighting at PDE nodes and injected at EDGE nodes;
// bilinear prolongation.  A coarse level represents the hole only to its own spacing, and
// the coarse-grid correction is poor in the layer between the fine and the coarse hole
// edges: after each correction a band of a few nodes around the hole is relaxed several
// times (one CTA), which restores the cycle's contraction (about 0.3 per V(2,2) cycle).
#include "../../include/helm.h"
#include "launch.h"
#include "pdl.cuh"
#include "fp_bits.cuh"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

namespace helm {
namespace {

constexpr int AN_NT = 256;
constexpr int AN_NC = 8;            // coarsest level (solved exactly)
constexpr int AN_BAND = 4;          // band half-width around the hole, in nodes of the level
constexpr int AN_BAND_SWEEPS = 4;
constexpr bool AN_BAND_SMEM = true;  // band sweeps in shared memory where the ring fits
constexpr bool AN_TILES = true;      // each side's sweeps of a level in one tile launch
constexpr bool AN_GRAPHS = true;     // an outer step replayed as one graph launch
constexpr size_t AN_SMEM_MAX = 227 * 1024;
enum : unsigned char { AN_PDE = 0, AN_EDGE = 1, AN_HOLE = 2 };

template <typename R> struct CX;
template <> struct CX<float> { typedef float2 T; };
template <> struct CX<double> { typedef double2 T; };

__host__ __device__ constexpr size_t an_a16(size_t b) { return (b + 15) & ~(size_t)15; }

int grid_for(long work) { return (int)std::min<long>((work + AN_NT - 1) / AN_NT, 152L * 16); }

// mean of the inward neighbours of an edge node (two at a corner)
template <typename T>
__device__ __forceinline__ T inward_mean(const T* e, int i, int j, int n)
{
    const int S = n + 1;
    T s;
    s.x = 0;
    s.y = 0;
    int c = 0;
    if (i == 0) { s.x += e[S + j].x; s.y += e[S + j].y; ++c; }
    if (i == n) { s.x += e[(n - 1) * S + j].x; s.y += e[(n - 1) * S + j].y; ++c; }
    if (j == 0) { s.x += e[i * S + 1].x; s.y += e[i * S + 1].y; ++c; }
    if (j == n) { s.x += e[i * S + n - 1].x; s.y += e[i * S + n - 1].y; ++c; }
    if (c == 2) { s.x *= 0.5f; s.y *= 0.5f; }
    return s;
}

// sum of the non-hole neighbours of a PDE node (hole entries of an iterate are zero)
template <typename T>
__device__ __forceinline__ T nbr_sum(const T* e, int q, int S)
{
    T a = e[q - S], b = e[q + S], c = e[q - 1], d = e[q + 1];
    T s;
    s.x = (a.x + b.x) + (c.x + d.x);
    s.y = (a.y + b.y) + (c.y + d.y);
    return s;
}

// Red-black Gauss-Seidel over the box [i0, i1] x [j0, j1] for nodes of colour (i + j) & 1;
// PDE rows e = (sum of neighbours - h^2 rhs) / (4 + sigma h^2), EDGE rows e = mean of the
// inward neighbours + h rhs.  pde_only: the band sweeps near the hole.
template <typename R>
__global__ void __launch_bounds__(AN_NT)
k_an_rbgs(typename CX<R>::T* __restrict__ e, const typename CX<R>::T* __restrict__ rhs,
          const unsigned char* __restrict__ typ, int n, R h, R dinv, int color, int i0, int i1, int j0,
          int j1)
{
    typedef typename CX<R>::T c2;
    const int S = n + 1;
    const int half = (j1 - j0 + 2) / 2;
    const long total = (long)(i1 - i0 + 1) * half;
    const R h2 = h * h;
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
        const int i = i0 + (int)(t / half);
        const int j = j0 + (((i + j0) & 1) ^ color) + 2 * (int)(t % half);
        if (j > j1) continue;
        const int q = i * S + j;
        const unsigned char ty = typ[q];
        if (ty == AN_PDE) {
            const c2 s = nbr_sum(e, q, S);
            const c2 r = rhs[q];
            c2 v;
            v.x = (s.x - h2 * r.x) * dinv;
            v.y = (s.y - h2 * r.y) * dinv;
            e[q] = v;
        } else if (ty == AN_EDGE) {
            const c2 m = inward_mean(e, i, j, n);
            const c2 r = rhs[q];
            c2 v;
            v.x = m.x + h * r.x;
            v.y = m.y + h * r.y;
            e[q] = v;
        }
    }
}

// One CTA: `sweeps` red-black sweeps over the PDE nodes of the ring [b0, b1]^2 minus the
// hole's index box [lo, hi]^2, through L2 (loads bypass L1 so that each half-sweep sees the
// CTA's previous writes).
template <typename R>
__global__ void __launch_bounds__(1024)
k_an_band(typename CX<R>::T* e, const typename CX<R>::T* __restrict__ rhs, const unsigned char* __restrict__ typ,
          int n, R h, R dinv, int b0, int b1, int lo, int hi, int sweeps)
{
    typedef typename CX<R>::T c2;
    const int S = n + 1;
    const int w = b1 - b0 + 1, th = lo - b0, bh = b1 - hi, hh = hi - lo + 1;
    const int nA = th * w, nB = bh * w, nC = hh * th, nD = hh * bh;
    const int total = nA + nB + nC + nD;
    const R h2 = h * h;
    for (int s = 0; s < 2 * sweeps; ++s) {
        const int color = s & 1;
        for (int t = threadIdx.x; t < total; t += blockDim.x) {
            int i, j;
            if (t < nA) { i = b0 + t / w; j = b0 + t % w; }
            else if (t < nA + nB) { const int u = t - nA; i = hi + 1 + u / w; j = b0 + u % w; }
            else if (t < nA + nB + nC) { const int u = t - nA - nB; i = lo + u / th; j = b0 + u % th; }
            else { const int u = t - nA - nB - nC; i = lo + u / bh; j = hi + 1 + u % bh; }
            if (((i + j) & 1) != color) continue;
            const int q = i * S + j;
            if (typ[q] != AN_PDE) continue;
            const c2 a = __ldcg(e + q - S), b = __ldcg(e + q + S), c = __ldcg(e + q - 1), d = __ldcg(e + q + 1);
            const c2 r = rhs[q];
            c2 v;
            v.x = (((a.x + b.x) + (c.x + d.x)) - h2 * r.x) * dinv;
            v.y = (((a.y + b.y) + (c.y + d.y)) - h2 * r.y) * dinv;
            __stcg(e + q, v);
        }
        __syncthreads();
    }
}

// The same sweeps with the ring and a 1-node halo around it staged in shared memory: the
// ring's four strips (rows b0 - 1 .. lo - 1 and hi + 1 .. b1 + 1 across the band's width
// plus halo; columns b0 - 1 .. lo - 1 and hi + 1 .. b1 + 1 over the hole's rows); nodes
// of the hole's box read as zero, as they hold in the iterate.  The ring's rhs is staged
// by ring index.
struct AnRing {
    int b0, b1, lo, hi;
    int w, th, bh, hh, W2, sA, sB, sC, sD, nA, nB, nC, nD;
    __host__ __device__ AnRing(int b0_, int b1_, int lo_, int hi_) : b0(b0_), b1(b1_), lo(lo_), hi(hi_)
    {
        w = b1 - b0 + 1;
        th = lo - b0;
        bh = b1 - hi;
        hh = hi - lo + 1;
        W2 = w + 2;
        sA = (th + 1) * W2;
        sB = (bh + 1) * W2;
        sC = hh * (th + 1);
        sD = hh * (bh + 1);
        nA = th * w;
        nB = bh * w;
        nC = hh * th;
        nD = hh * bh;
    }
    __host__ __device__ int stored() const { return sA + sB + sC + sD; }
    __host__ __device__ int total() const { return nA + nB + nC + nD; }
    // shared-memory slot of node (i, j) of the window, -1 inside the hole's box
    __device__ int slot(int i, int j) const
    {
        if (i < lo) return (i - (b0 - 1)) * W2 + (j - (b0 - 1));
        if (i > hi) return sA + (i - (hi + 1)) * W2 + (j - (b0 - 1));
        if (j < lo) return sA + sB + (i - lo) * (th + 1) + (j - (b0 - 1));
        if (j > hi) return sA + sB + sC + (i - lo) * (bh + 1) + (j - (hi + 1));
        return -1;
    }
    // node of window slot u
    __device__ void window_node(int u, int& i, int& j) const
    {
        if (u < sA) { i = b0 - 1 + u / W2; j = b0 - 1 + u % W2; return; }
        u -= sA;
        if (u < sB) { i = hi + 1 + u / W2; j = b0 - 1 + u % W2; return; }
        u -= sB;
        if (u < sC) { i = lo + u / (th + 1); j = b0 - 1 + u % (th + 1); return; }
        u -= sC;
        i = lo + u / (bh + 1);
        j = hi + 1 + u % (bh + 1);
    }
    // node of ring index t (the order of k_an_band)
    __device__ void ring_node(int t, int& i, int& j) const
    {
        if (t < nA) { i = b0 + t / w; j = b0 + t % w; return; }
        t -= nA;
        if (t < nB) { i = hi + 1 + t / w; j = b0 + t % w; return; }
        t -= nB;
        if (t < nC) { i = lo + t / th; j = b0 + t % th; return; }
        t -= nC;
        i = lo + t / bh;
        j = hi + 1 + t % bh;
    }
};

template <typename R>
size_t an_band_bytes(const AnRing& g)
{
    const size_t c = sizeof(typename CX<R>::T);
    return (size_t)g.stored() * c + (size_t)g.total() * c;
}

// Each thread owns ring indices threadIdx.x + 1024 k (k < AN_BAND_PT) and keeps, for each,
// the shared-memory slots of the node and of its four neighbours (-1: the hole's box),
// found once; a half-sweep is then shared-memory loads and the update alone.
constexpr int AN_BAND_PT = 5;

template <typename R>
__global__ void __launch_bounds__(1024)
k_an_band_s(typename CX<R>::T* __restrict__ e, const typename CX<R>::T* __restrict__ rhs,
            const unsigned char* __restrict__ typ, int n, R h, R dinv, AnRing g, int sweeps)
{
    typedef typename CX<R>::T c2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int S = n + 1;
    const int stored = g.stored(), total = g.total();
    c2* Es = reinterpret_cast<c2*>(smem_raw);
    c2* Rs = Es + stored;
    for (int u = threadIdx.x; u < stored; u += blockDim.x) {
        int i, j;
        g.window_node(u, i, j);
        Es[u] = e[i * S + j];
    }
    int self[AN_BAND_PT], nb[AN_BAND_PT][4];
    unsigned colour = 0;                          // bit k: the owned node's colour
#pragma unroll
    for (int k = 0; k < AN_BAND_PT; ++k) {
        const int t = threadIdx.x + 1024 * k;
        self[k] = -1;
        nb[k][0] = nb[k][1] = nb[k][2] = nb[k][3] = -1;
        if (t < total) {
            int i, j;
            g.ring_node(t, i, j);
            Rs[t] = rhs[i * S + j];
            if (typ[i * S + j] == AN_PDE) {
                self[k] = g.slot(i, j);
                nb[k][0] = g.slot(i - 1, j);
                nb[k][1] = g.slot(i + 1, j);
                nb[k][2] = g.slot(i, j - 1);
                nb[k][3] = g.slot(i, j + 1);
                colour |= (unsigned)((i + j) & 1) << k;
            }
        }
    }
    __syncthreads();
    const R h2 = h * h;
    c2 z;
    z.x = 0;
    z.y = 0;
    for (int s = 0; s < 2 * sweeps; ++s) {
        const unsigned color = s & 1;
#pragma unroll
        for (int k = 0; k < AN_BAND_PT; ++k) {
            if (self[k] < 0 || ((colour >> k) & 1u) != color) continue;
            const c2 a = nb[k][0] < 0 ? z : Es[nb[k][0]], b = nb[k][1] < 0 ? z : Es[nb[k][1]];
            const c2 c = nb[k][2] < 0 ? z : Es[nb[k][2]], d = nb[k][3] < 0 ? z : Es[nb[k][3]];
            const c2 r = Rs[threadIdx.x + 1024 * k];
            c2 v;
            v.x = (((a.x + b.x) + (c.x + d.x)) - h2 * r.x) * dinv;
            v.y = (((a.y + b.y) + (c.y + d.y)) - h2 * r.y) * dinv;
            Es[self[k]] = v;
        }
        __syncthreads();
    }
#pragma unroll
    for (int k = 0; k < AN_BAND_PT; ++k) {
        const int t = threadIdx.x + 1024 * k;
        if (self[k] < 0) continue;
        int i, j;
        g.ring_node(t, i, j);
        e[i * S + j] = Es[self[k]];
    }
}

// residual of the level's row at a fine node (zero on the hole)
template <typename R>
__device__ __forceinline__ typename CX<R>::T an_resid(const typename CX<R>::T* e, const typename CX<R>::T* rhs,
                                                      const unsigned char* typ, int i, int j, int n, R h, R sig,
                                                      bool zero)
{
    typedef typename CX<R>::T c2;
    const int S = n + 1, q = i * S + j;
    const unsigned char ty = typ[q];
    c2 r = rhs[q];
    if (ty == AN_HOLE) { r.x = 0; r.y = 0; return r; }
    if (zero) return r;
    const c2 c = e[q];
    if (ty == AN_PDE) {
        const c2 s = nbr_sum(e, q, S);
        const R ih2 = (R)1 / (h * h);
        r.x -= (s.x - (R)4 * c.x) * ih2 - sig * c.x;
        r.y -= (s.y - (R)4 * c.y) * ih2 - sig * c.y;
    } else {
        const c2 m = inward_mean(e, i, j, n);
        r.x -= (c.x - m.x) / h;
        r.y -= (c.y - m.y) / h;
    }
    return r;
}

// ---------------------------------------------------------------------------
// Tile kernels: a level's sweeps (and its residual + restriction) on a window in shared
// memory, so that the sweeps of one side of the cycle are one launch
// ---------------------------------------------------------------------------
// A window [sy0, sy1] x [sx0, sx1] of the level (clipped to [0, n]) is staged with row
// stride SW.  Half-sweep k updates the nodes of its colour that lie k + 1 nodes inside
// every window side that is not a side of the grid, so that each updated node sees the
// values the per-level kernels would give it; after 2 nu half-sweeps the values are those
// of the per-level sweeps on the window shrunk by 2 nu (grid sides excepted).
constexpr int AN_CT = 16;            // coarse nodes per side of a descent tile
constexpr int AN_FT = 32;            // fine nodes per side of an ascent tile

// mean of the inward neighbours of edge node (i, j) at window index q
template <typename T>
__device__ __forceinline__ T inward_mean_w(const T* e, int q, int SW, int i, int j, int n)
{
    T s;
    s.x = 0;
    s.y = 0;
    int c = 0;
    if (i == 0) { s.x += e[q + SW].x; s.y += e[q + SW].y; ++c; }
    if (i == n) { s.x += e[q - SW].x; s.y += e[q - SW].y; ++c; }
    if (j == 0) { s.x += e[q + 1].x; s.y += e[q + 1].y; ++c; }
    if (j == n) { s.x += e[q - 1].x; s.y += e[q - 1].y; ++c; }
    if (c == 2) { s.x *= 0.5f; s.y *= 0.5f; }
    return s;
}

template <typename R>
__device__ __forceinline__ typename CX<R>::T an_resid_w(const typename CX<R>::T* e, const typename CX<R>::T* rhs,
                                                        const unsigned char* typ, int q, int SW, int i, int j,
                                                        int n, R h, R sig, bool zero)
{
    typedef typename CX<R>::T c2;
    const unsigned char ty = typ[q];
    c2 r = rhs[q];
    if (ty == AN_HOLE) { r.x = 0; r.y = 0; return r; }
    if (zero) return r;
    const c2 c = e[q];
    if (ty == AN_PDE) {
        const c2 s = nbr_sum(e, q, SW);
        const R ih2 = (R)1 / (h * h);
        r.x -= (s.x - (R)4 * c.x) * ih2 - sig * c.x;
        r.y -= (s.y - (R)4 * c.y) * ih2 - sig * c.y;
    } else {
        const c2 m = inward_mean_w(e, q, SW, i, j, n);
        r.x -= (c.x - m.x) / h;
        r.y -= (c.y - m.y) / h;
    }
    return r;
}

struct AnWin {
    int sx0, sx1, sy0, sy1, SW;
};

// stage e (or zeros), rhs and the row types of the window
template <typename R>
__device__ void an_stage(typename CX<R>::T* E, typename CX<R>::T* Rr, unsigned char* Ty, const AnWin& w,
                         const typename CX<R>::T* __restrict__ e, const typename CX<R>::T* __restrict__ rhs,
                         const unsigned char* __restrict__ typ, int n, bool load_e)
{
    typedef typename CX<R>::T c2;
    const int S = n + 1, ww = w.sx1 - w.sx0 + 1, wh = w.sy1 - w.sy0 + 1;
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    c2 z;
    z.x = 0;
    z.y = 0;
    for (int ly = threadIdx.x >> 5; ly < wh; ly += nw)
        for (int lx = lane; lx < ww; lx += 32) {
            const int g = (w.sy0 + ly) * S + w.sx0 + lx, q = ly * w.SW + lx;
            E[q] = load_e ? e[g] : z;
            Rr[q] = rhs[g];
            Ty[q] = typ[g];
        }
}

// Red-black Gauss-Seidel on the nodes of colour `color` in row i, columns ux0..ux1, of
// arrays with row stride SW whose element 0 is node (oy, ox); the warp's lanes take the
// row's nodes of that colour.  PDE rows take the 5-point local solve, EDGE rows the mean
// of their inward neighbours plus h rhs.
template <typename R>
__device__ __forceinline__ void an_row(typename CX<R>::T* E, const typename CX<R>::T* Rr, const unsigned char* Ty,
                                       int SW, int oy, int ox, int i, int ux0, int ux1, int n, R h, R dinv,
                                       int color)
{
    typedef typename CX<R>::T c2;
    const R h2 = h * h;
    const int jf = ux0 + ((i + ux0 + color) & 1);
    for (int j = jf + 2 * (int)(threadIdx.x & 31); j <= ux1; j += 64) {
        const int q = (i - oy) * SW + (j - ox);
        const unsigned char ty = Ty[q];
        if (ty == AN_PDE) {
            const c2 sn = nbr_sum(E, q, SW);
            const c2 r = Rr[q];
            c2 v;
            v.x = (sn.x - h2 * r.x) * dinv;
            v.y = (sn.y - h2 * r.y) * dinv;
            E[q] = v;
        } else if (ty == AN_EDGE) {
            const c2 m = inward_mean_w(E, q, SW, i, j, n);
            const c2 r = Rr[q];
            c2 v;
            v.x = m.x + h * r.x;
            v.y = m.y + h * r.y;
            E[q] = v;
        }
    }
}

// one half-sweep over rows uy0..uy1, a warp per row
template <typename R>
__device__ __forceinline__ void an_half(typename CX<R>::T* E, const typename CX<R>::T* Rr, const unsigned char* Ty,
                                        int SW, int oy, int ox, int uy0, int uy1, int ux0, int ux1, int n, R h,
                                        R dinv, int color)
{
    const int nw = blockDim.x >> 5;
    for (int i = uy0 + (int)(threadIdx.x >> 5); i <= uy1; i += nw)
        an_row<R>(E, Rr, Ty, SW, oy, ox, i, ux0, ux1, n, h, dinv, color);
}

// Full weighting of the residual at coarse PDE nodes, injection at EDGE nodes, zero on the
// hole, for coarse rows CI0..CI1, columns CJ0..CJ1; Res holds the fine residual with row
// stride RW, element 0 at fine node (roy, rox).  The coarse value goes to out(I, J).
template <typename R, typename F>
__device__ __forceinline__ void an_restrict_res(const typename CX<R>::T* Res, int RW, int roy, int rox,
                                                const unsigned char* tc, int Sc, int CI0, int CI1, int CJ0, int CJ1,
                                                F out)
{
    typedef typename CX<R>::T c2;
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int I = CI0 + (threadIdx.x >> 5); I <= CI1; I += nw)
        for (int J = CJ0 + lane; J <= CJ1; J += 32) {
            const unsigned char ty = tc[I * Sc + J];
            c2 v;
            if (ty == AN_HOLE) {
                v.x = 0;
                v.y = 0;
            } else if (ty == AN_EDGE) {
                v = Res[(2 * I - roy) * RW + (2 * J - rox)];
            } else {
                R ax = 0, ay = 0;
#pragma unroll
                for (int a = -1; a <= 1; ++a)
#pragma unroll
                    for (int b = -1; b <= 1; ++b) {
                        const R wgt = (R)((2 - (a < 0 ? -a : a)) * (2 - (b < 0 ? -b : b)));
                        const c2 r = Res[(2 * I + a - roy) * RW + (2 * J + b - rox)];
                        ax += wgt * r.x;
                        ay += wgt * r.y;
                    }
                v.x = ax * (R)(1.0 / 16.0);
                v.y = ay * (R)(1.0 / 16.0);
            }
            out(I, J, v);
        }
}

// nu red-black sweeps on the window
template <typename R>
__device__ void an_sweeps_w(typename CX<R>::T* E, const typename CX<R>::T* Rr, const unsigned char* Ty,
                            const AnWin& w, int n, R h, R dinv, int nu)
{
    for (int k = 0; k < 2 * nu; ++k) {
        const int ux0 = w.sx0 == 0 ? 0 : w.sx0 + k + 1, ux1 = w.sx1 == n ? n : w.sx1 - k - 1;
        const int uy0 = w.sy0 == 0 ? 0 : w.sy0 + k + 1, uy1 = w.sy1 == n ? n : w.sy1 - k - 1;
        an_half<R>(E, Rr, Ty, w.SW, w.sy0, w.sx0, uy0, uy1, ux0, ux1, n, h, dinv, k & 1);
        __syncthreads();
    }
}

template <typename R>
__host__ __device__ size_t an_win_bytes(int SW)
{
    const size_t pts = (size_t)SW * SW;
    return 2 * an_a16(pts * sizeof(typename CX<R>::T)) + an_a16(pts);
}
__host__ __device__ constexpr int an_down_sw(int nu1) { return 2 * AN_CT + 3 + 4 * nu1; }
constexpr int AN_RW = 2 * AN_CT + 1;  // fine residual rows / columns of a descent tile
template <typename R>
size_t an_down_bytes(int nu1)
{
    return an_win_bytes<R>(an_down_sw(nu1)) + an_a16((size_t)AN_RW * AN_RW * sizeof(typename CX<R>::T));
}
__host__ __device__ constexpr int an_up_sw(int nu2) { return AN_FT + 4 * nu2; }

// Descent of one level: nu1 sweeps, then the coarse rhs (full weighting of the residual at
// coarse PDE nodes, injection at coarse edge nodes, zero on the hole) and a zero coarse
// iterate for the coarse nodes [I0, I0 + AN_CT) x [J0, J0 + AN_CT); the swept fine iterate
// goes to e_out on the fine nodes [2 I0, 2 I0 + 2 AN_CT) x [2 J0, 2 J0 + 2 AN_CT): a
// separate buffer, since other CTAs stage their windows from e_in meanwhile.
template <typename R>
__global__ void __launch_bounds__(AN_NT)
k_an_down(const typename CX<R>::T* __restrict__ e, typename CX<R>::T* __restrict__ e_out,
          const typename CX<R>::T* __restrict__ rhs,
          const unsigned char* __restrict__ typ, int n, R h, R dinv, R sig, int nu1, int load_e,
          typename CX<R>::T* __restrict__ rc, typename CX<R>::T* __restrict__ ec,
          const unsigned char* __restrict__ tc, int nc)
{
    typedef typename CX<R>::T c2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int ntc = (nc + AN_CT) / AN_CT;
    const int I0 = (blockIdx.x / ntc) * AN_CT, J0 = (blockIdx.x % ntc) * AN_CT;
    const int hw = 2 + 2 * nu1;               // low side; the high side needs 2 nu1
    AnWin w;
    w.SW = an_down_sw(nu1);
    w.sy0 = max(0, 2 * I0 - hw);
    w.sy1 = min(n, 2 * I0 + 2 * AN_CT + 2 * nu1);
    w.sx0 = max(0, 2 * J0 - hw);
    w.sx1 = min(n, 2 * J0 + 2 * AN_CT + 2 * nu1);
    const size_t pts = (size_t)w.SW * w.SW;
    c2* E = reinterpret_cast<c2*>(smem_raw);
    c2* Rr = reinterpret_cast<c2*>(smem_raw + an_a16(pts * sizeof(c2)));
    unsigned char* Ty = smem_raw + 2 * an_a16(pts * sizeof(c2));
    c2* Res = reinterpret_cast<c2*>(smem_raw + an_win_bytes<R>(w.SW));
    an_stage<R>(E, Rr, Ty, w, e, rhs, typ, n, load_e != 0);
    __syncthreads();
    an_sweeps_w<R>(E, Rr, Ty, w, n, h, dinv, nu1);
    const bool zero = nu1 == 0 && load_e == 0;
    const int Sc = nc + 1, S = n + 1;
    const int ci1 = min(nc, I0 + AN_CT - 1), cj1 = min(nc, J0 + AN_CT - 1);
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    // the fine residual once per node: rows / columns 2 I0 - 1 .. 2 ci1 + 1 (within the grid)
    const int roy = 2 * I0 - 1, rox = 2 * J0 - 1;
    {
        const int ry0 = max(0, roy), ry1 = min(n, 2 * ci1 + 1), rx0 = max(0, rox), rx1 = min(n, 2 * cj1 + 1);
        for (int i = ry0 + (threadIdx.x >> 5); i <= ry1; i += nw)
            for (int j = rx0 + lane; j <= rx1; j += 32)
                Res[(i - roy) * AN_RW + (j - rox)] =
                    an_resid_w<R>(E, Rr, Ty, (i - w.sy0) * w.SW + (j - w.sx0), w.SW, i, j, n, h, sig, zero);
    }
    __syncthreads();
    an_restrict_res<R>(Res, AN_RW, roy, rox, tc, Sc, I0, ci1, J0, cj1, [&](int I, int J, c2 v) {
        c2 z;
        z.x = 0;
        z.y = 0;
        ec[I * Sc + J] = z;
        rc[I * Sc + J] = v;
    });
    {
        const int fi1 = min(n, 2 * I0 + 2 * AN_CT - 1), fj1 = min(n, 2 * J0 + 2 * AN_CT - 1);
        for (int i = 2 * I0 + (threadIdx.x >> 5); i <= fi1; i += nw)
            for (int j = 2 * J0 + lane; j <= fj1; j += 32) e_out[i * S + j] = E[(i - w.sy0) * w.SW + (j - w.sx0)];
    }
}

// Ascent sweeps of one level: nu2 sweeps of e_in; the fine nodes [32 by, 32 by + 32) x
// [32 bx, 32 bx + 32) go to e_out.
template <typename R>
__global__ void __launch_bounds__(AN_NT)
k_an_up(const typename CX<R>::T* __restrict__ e, typename CX<R>::T* __restrict__ e_out,
        const typename CX<R>::T* __restrict__ rhs,
        const unsigned char* __restrict__ typ, int n, R h, R dinv, int nu2)
{
    typedef typename CX<R>::T c2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nt = (n + AN_FT) / AN_FT;
    const int i0 = (blockIdx.x / nt) * AN_FT, j0 = (blockIdx.x % nt) * AN_FT;
    const int hw = 2 * nu2;
    AnWin w;
    w.SW = an_up_sw(nu2);
    w.sy0 = max(0, i0 - hw);
    w.sy1 = min(n, i0 + AN_FT - 1 + hw);
    w.sx0 = max(0, j0 - hw);
    w.sx1 = min(n, j0 + AN_FT - 1 + hw);
    const size_t pts = (size_t)w.SW * w.SW;
    c2* E = reinterpret_cast<c2*>(smem_raw);
    c2* Rr = reinterpret_cast<c2*>(smem_raw + an_a16(pts * sizeof(c2)));
    unsigned char* Ty = smem_raw + 2 * an_a16(pts * sizeof(c2));
    an_stage<R>(E, Rr, Ty, w, e, rhs, typ, n, true);
    __syncthreads();
    an_sweeps_w<R>(E, Rr, Ty, w, n, h, dinv, nu2);
    const int S = n + 1, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int fi1 = min(n, i0 + AN_FT - 1), fj1 = min(n, j0 + AN_FT - 1);
    for (int i = i0 + (threadIdx.x >> 5); i <= fi1; i += nw)
        for (int j = j0 + lane; j <= fj1; j += 32) e_out[i * S + j] = E[(i - w.sy0) * w.SW + (j - w.sx0)];
}

// coarse rhs: full weighting of the fine residual at PDE nodes, injection at EDGE nodes;
// coarse iterate := 0
template <typename R>
__global__ void __launch_bounds__(AN_NT)
k_an_restrict(const typename CX<R>::T* __restrict__ ef, const typename CX<R>::T* __restrict__ rf,
              const unsigned char* __restrict__ tf, int nf, R hf, R sig, typename CX<R>::T* __restrict__ rc,
              typename CX<R>::T* __restrict__ ec, const unsigned char* __restrict__ tc, int nc, int zero)
{
    typedef typename CX<R>::T c2;
    const int Sc = nc + 1;
    const long total = (long)Sc * Sc;
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
        const int I = (int)(t / Sc), J = (int)(t % Sc);
        c2 z;
        z.x = 0;
        z.y = 0;
        ec[t] = z;
        const unsigned char ty = tc[t];
        if (ty == AN_HOLE) {
            rc[t] = z;
        } else if (ty == AN_EDGE) {
            rc[t] = an_resid<R>(ef, rf, tf, 2 * I, 2 * J, nf, hf, sig, zero != 0);
        } else {
            R ax = 0, ay = 0;
#pragma unroll
            for (int a = -1; a <= 1; ++a)
#pragma unroll
                for (int b = -1; b <= 1; ++b) {
                    const R wgt = (R)((2 - (a < 0 ? -a : a)) * (2 - (b < 0 ? -b : b)));
                    const c2 r = an_resid<R>(ef, rf, tf, 2 * I + a, 2 * J + b, nf, hf, sig, zero != 0);
                    ax += wgt * r.x;
                    ay += wgt * r.y;
                }
            c2 v;
            v.x = ax * (R)(1.0 / 16.0);
            v.y = ay * (R)(1.0 / 16.0);
            rc[t] = v;
        }
    }
}

// fine iterate += bilinear interpolation of the coarse one (fine hole nodes untouched)
template <typename R>
__global__ void __launch_bounds__(AN_NT)
k_an_prolong(const typename CX<R>::T* __restrict__ ec, int nc, typename CX<R>::T* __restrict__ ef,
             const unsigned char* __restrict__ tf, int nf)
{
    typedef typename CX<R>::T c2;
    const int Sf = nf + 1, Sc = nc + 1;
    const long total = (long)Sf * Sf;
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
        if (tf[t] == AN_HOLE) continue;
        const int i = (int)(t / Sf), j = (int)(t % Sf);
        const int I0 = i >> 1, I1 = (i + 1) >> 1, J0 = j >> 1, J1 = (j + 1) >> 1;
        const c2 a = ec[I0 * Sc + J0], b = ec[I1 * Sc + J0], c = ec[I0 * Sc + J1], d = ec[I1 * Sc + J1];
        c2 v = ef[t];
        v.x += (R)0.25 * (((a.x + b.x) + c.x) + d.x);
        v.y += (R)0.25 * (((a.y + b.y) + c.y) + d.y);
        ef[t] = v;
    }
}

// coarsest level: e = Ainv rhs over its m unknowns (map: unknown -> node); a warp per row,
// its lanes over the columns (coalesced rows of Ainv), partial sums added by a butterfly
template <typename R>
__device__ __forceinline__ void an_dense_solve(const typename CX<R>::T* rhs, typename CX<R>::T* e,
                                               const double* __restrict__ Ainv, const int* __restrict__ map, int m)
{
    typedef typename CX<R>::T c2;
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int r = threadIdx.x >> 5; r < m; r += nw) {
        double ax = 0.0, ay = 0.0;
        for (int c = lane; c < m; c += 32) {
            const double a = Ainv[(size_t)r * m + c];
            const c2 v = rhs[map[c]];
            ax += a * (double)v.x;
            ay += a * (double)v.y;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            ax += __shfl_xor_sync(0xffffffffu, ax, o);
            ay += __shfl_xor_sync(0xffffffffu, ay, o);
        }
        if (lane == 0) {
            c2 v;
            v.x = (R)ax;
            v.y = (R)ay;
            e[map[r]] = v;
        }
    }
}

template <typename R>
__global__ void __launch_bounds__(AN_NT)
k_an_coarse(const typename CX<R>::T* __restrict__ rhs, typename CX<R>::T* __restrict__ e,
            const double* __restrict__ Ainv, const int* __restrict__ map, int m)
{
    an_dense_solve<R>(rhs, e, Ainv, map, m);
}

// ---------------------------------------------------------------------------
// Coarse tail: the coarsest levels in one CTA, in shared memory
// ---------------------------------------------------------------------------
// The same V-cycle as the per-level kernels (sweeps, restriction, prolongation, band
// sweeps, exact coarsest level), with block-wide barriers between its phases instead of
// kernel boundaries.  Levels 64, 32, 16, 8 hold about 5.7 K nodes.  In FP64 one SM's
// arithmetic rate (a small fraction of its FP32 rate) makes the level-64 restriction slower
// in one CTA than spread over several, so the FP64 tail starts lower.
constexpr int AN_TAIL_TOP_F = 64;
constexpr int AN_TAIL_TOP_D = 16;
constexpr int AN_TAIL_MAX = 4;

struct AnTailLev {
    int n, b0, b1, lo, hi;
    double h, dinv;
    const unsigned char* typ;
};
struct AnTail {
    int L, nu1, nu2, load_e, m;
    double sigma;
    AnTailLev lev[AN_TAIL_MAX];
    const double* Ainv;
    const int* map;
};


template <typename R>
__global__ void __launch_bounds__(1024, 1)
k_an_tail(typename CX<R>::T* __restrict__ eg, const typename CX<R>::T* __restrict__ rg, AnTail T)
{
    typedef typename CX<R>::T c2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    c2* E[AN_TAIL_MAX];
    c2* Rr[AN_TAIL_MAX];
    unsigned char* Ty[AN_TAIL_MAX];
    size_t off = 0;
    for (int l = 0; l < T.L; ++l) {
        const size_t pts = (size_t)(T.lev[l].n + 1) * (T.lev[l].n + 1);
        E[l] = reinterpret_cast<c2*>(smem_raw + off);
        off += an_a16(pts * sizeof(c2));
        Rr[l] = reinterpret_cast<c2*>(smem_raw + off);
        off += an_a16(pts * sizeof(c2));
        Ty[l] = smem_raw + off;
        off += an_a16(pts);
    }
    c2* Res = reinterpret_cast<c2*>(smem_raw + off);     // the top level's residual, once per node
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int l = 0; l < T.L; ++l) {
        const int pts = (T.lev[l].n + 1) * (T.lev[l].n + 1);
        for (int q = threadIdx.x; q < pts; q += blockDim.x) Ty[l][q] = T.lev[l].typ[q];
    }
    {
        const int pts = (T.lev[0].n + 1) * (T.lev[0].n + 1);
        c2 z;
        z.x = 0;
        z.y = 0;
        for (int q = threadIdx.x; q < pts; q += blockDim.x) {
            Rr[0][q] = rg[q];
            E[0][q] = T.load_e ? eg[q] : z;
        }
    }
    __syncthreads();
    const R sig = (R)T.sigma;
    // descent
    for (int l = 0; l + 1 < T.L; ++l) {
        const AnTailLev& Lv = T.lev[l];
        const R h = (R)Lv.h, dinv = (R)Lv.dinv;
        const int n = Lv.n, S = n + 1;
        for (int k = 0; k < 2 * T.nu1; ++k) {
            an_half<R>(E[l], Rr[l], Ty[l], S, 0, 0, 0, n, 0, n, n, h, dinv, k & 1);
            __syncthreads();
        }
        const int nc = T.lev[l + 1].n, Sc = nc + 1;
        const bool zero = T.nu1 == 0 && (l > 0 || !T.load_e);
        for (int i = threadIdx.x >> 5; i <= n; i += nw)
            for (int j = lane; j <= n; j += 32)
                Res[i * S + j] = an_resid<R>(E[l], Rr[l], Ty[l], i, j, n, h, sig, zero);
        __syncthreads();
        c2* const Ec = E[l + 1];
        c2* const Rc = Rr[l + 1];
        an_restrict_res<R>(Res, S, 0, 0, Ty[l + 1], Sc, 0, nc, 0, nc, [&](int I, int J, c2 v) {
            c2 z;
            z.x = 0;
            z.y = 0;
            Ec[I * Sc + J] = z;
            Rc[I * Sc + J] = v;
        });
        __syncthreads();
    }
    // the coarsest level, exactly
    an_dense_solve<R>(Rr[T.L - 1], E[T.L - 1], T.Ainv, T.map, T.m);
    __syncthreads();
    // ascent
    for (int l = T.L - 2; l >= 0; --l) {
        const AnTailLev& Lv = T.lev[l];
        const int n = Lv.n, S = n + 1, nc = T.lev[l + 1].n, Sc = nc + 1;
        const R h = (R)Lv.h, dinv = (R)Lv.dinv;
        for (int i = threadIdx.x >> 5; i <= n; i += nw)
            for (int j = lane; j <= n; j += 32) {
                const int q = i * S + j;
                if (Ty[l][q] == AN_HOLE) continue;
                const int I0 = i >> 1, I1 = (i + 1) >> 1, J0 = j >> 1, J1 = (j + 1) >> 1;
                const c2 a = E[l + 1][I0 * Sc + J0], b = E[l + 1][I1 * Sc + J0];
                const c2 c = E[l + 1][I0 * Sc + J1], d = E[l + 1][I1 * Sc + J1];
                c2 v = E[l][q];
                v.x += (R)0.25 * (((a.x + b.x) + c.x) + d.x);
                v.y += (R)0.25 * (((a.y + b.y) + c.y) + d.y);
                E[l][q] = v;
            }
        __syncthreads();
        // band sweeps around the hole: rows b0..b1 of the ring [b0, b1]^2 minus [lo, hi]^2
        // (all PDE rows), a warp per row
        {
            const int b0 = Lv.b0, b1 = Lv.b1, lo = Lv.lo, hi = Lv.hi;
            for (int k = 0; k < 2 * AN_BAND_SWEEPS; ++k) {
                const int color = k & 1;
                for (int i = b0 + (threadIdx.x >> 5); i <= b1; i += nw) {
                    if (i < lo || i > hi) {
                        an_row<R>(E[l], Rr[l], Ty[l], S, 0, 0, i, b0, b1, n, h, dinv, color);
                    } else {
                        an_row<R>(E[l], Rr[l], Ty[l], S, 0, 0, i, b0, lo - 1, n, h, dinv, color);
                        an_row<R>(E[l], Rr[l], Ty[l], S, 0, 0, i, hi + 1, b1, n, h, dinv, color);
                    }
                }
                __syncthreads();
            }
        }
        for (int k = 0; k < 2 * T.nu2; ++k) {
            an_half<R>(E[l], Rr[l], Ty[l], S, 0, 0, 0, n, 0, n, n, h, dinv, k & 1);
            __syncthreads();
        }
    }
    const int pts = (T.lev[0].n + 1) * (T.lev[0].n + 1);
    for (int q = threadIdx.x; q < pts; q += blockDim.x) eg[q] = E[0][q];
}

template <typename R>
size_t an_tail_bytes(const int* ns, int L)
{
    size_t off = 0;
    for (int l = 0; l < L; ++l) {
        const size_t pts = (size_t)(ns[l] + 1) * (ns[l] + 1);
        off += 2 * an_a16(pts * sizeof(typename CX<R>::T)) + an_a16(pts);
    }
    return off + an_a16((size_t)(ns[0] + 1) * (ns[0] + 1) * sizeof(typename CX<R>::T));
}

// U := the hole data on hole nodes, 0 elsewhere (both iterate buffers)
__global__ void __launch_bounds__(AN_NT)
k_an_init(double2* __restrict__ U0, double2* __restrict__ U1, const double2* __restrict__ data,
          const unsigned char* __restrict__ typ, long total)
{
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
        const double2 v = (typ[t] == AN_HOLE) ? data[t] : make_double2(0.0, 0.0);
        U0[t] = v;
        U1[t] = v;
    }
}

// FP64 <-> inner precision; complex64's format changes run on the integer pipes
__device__ __forceinline__ double an_widen(float x) { return f2d_bits(x); }
__device__ __forceinline__ double an_widen(double x) { return x; }
__device__ __forceinline__ float an_narrow(double x, float) { return d2f_bits(x); }
__device__ __forceinline__ double an_narrow(double x, double) { return x; }

// U_out = U_in + e on the non-hole nodes (hole nodes keep the data in both buffers);
// per-block maxima of |e|^2 into part[2 b + 1]
template <typename R>
__global__ void __launch_bounds__(AN_NT)
k_an_update(const double2* __restrict__ Uin, double2* __restrict__ Uout, const typename CX<R>::T* __restrict__ e,
            const unsigned char* __restrict__ typ, long total, double* __restrict__ part)
{
    typedef typename CX<R>::T c2;
    R em = 0;
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
        if (typ[t] == AN_HOLE) continue;
        const c2 ev = e[t];
        double2 v = Uin[t];
        v.x += an_widen(ev.x);
        v.y += an_widen(ev.y);
        Uout[t] = v;
        const R a = ev.x * ev.x + ev.y * ev.y;
        em = em > a ? em : a;
    }
    __shared__ double sm[AN_NT / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const R x = __shfl_xor_sync(0xffffffffu, em, o);
        em = em > x ? em : x;
    }
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = (double)em;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = 0.0;
        for (int w = 0; w < AN_NT / 32; ++w) m = fmax(m, sm[w]);
        part[2 * blockIdx.x + 1] = m;
    }
}

// r = b - B U in FP64 (PDE: f - (Delta_h U + k^2 U); EDGE: q - (dU/dn - i k U)), stored,
// rounded to the inner precision, as the next rhs; per-block sums of |r|^2 (of the stored
// r) into part[2 b]
template <typename R>
__global__ void __launch_bounds__(AN_NT)
k_an_resid(const double2* __restrict__ U, const double2* __restrict__ data, const unsigned char* __restrict__ typ,
           typename CX<R>::T* __restrict__ rhs, int n, double h, double k2, double k, double* __restrict__ part)
{
    typedef typename CX<R>::T c2;
    const int S = n + 1;
    const long total = (long)S * S;
    const double ih2 = 1.0 / (h * h), ih = 1.0 / h;
    R r2 = 0;
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
        const unsigned char ty = typ[t];
        if (ty == AN_HOLE) continue;
        const int q = (int)t, i = q / S, j = q % S;
        const double2 c = U[q];
        const double2 dv = data[q];
        double2 r;
        if (ty == AN_PDE) {
            const double2 a = U[q - S], b = U[q + S], cc = U[q - 1], d = U[q + 1];
            r.x = dv.x - (((a.x + b.x) + (cc.x + d.x) - 4.0 * c.x) * ih2 + k2 * c.x);
            r.y = dv.y - (((a.y + b.y) + (cc.y + d.y) - 4.0 * c.y) * ih2 + k2 * c.y);
        } else {
            const double2 m = inward_mean(U, i, j, n);
            // dU/dn - i k U = (U - mean) / h + (k U.y, -k U.x)
            r.x = dv.x - ((c.x - m.x) * ih + k * c.y);
            r.y = dv.y - ((c.y - m.y) * ih - k * c.x);
        }
        c2 ri;
        ri.x = an_narrow(r.x, R());
        ri.y = an_narrow(r.y, R());
        rhs[q] = ri;
        r2 += ri.x * ri.x + ri.y * ri.y;
    }
    __shared__ double sa[AN_NT / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r2 += __shfl_xor_sync(0xffffffffu, r2, o);
    if ((threadIdx.x & 31) == 0) sa[threadIdx.x >> 5] = (double)r2;
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0;
        for (int w = 0; w < AN_NT / 32; ++w) a += sa[w];
        part[2 * blockIdx.x] = a;
    }
}

// real part of U -> out (double), and min over PDE nodes of (-L + sqrt(L^2 + 4 E)) / (2 E)
// (positive doubles order as their bit patterns)
__global__ void __launch_bounds__(AN_NT)
k_an_real(const double2* __restrict__ U, double* __restrict__ out, long total)
{
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x)
        out[t] = U[t].x;
}

__global__ void __launch_bounds__(AN_NT)
k_an_kstar(const double* __restrict__ E, const double* __restrict__ L, const unsigned char* __restrict__ typ,
           long total, unsigned long long* __restrict__ out)
{
    double best = 1e300;
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
        if (typ[t] != AN_PDE) continue;
        const double e = E[t], l = L[t];
        if (!(e > 0.0)) continue;
        best = fmin(best, (-l + sqrt(l * l + 4.0 * e)) / (2.0 * e));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) best = fmin(best, __shfl_xor_sync(0xffffffffu, best, o));
    if ((threadIdx.x & 31) == 0 && best < 1e300) atomicMin(out, (unsigned long long)__double_as_longlong(best));
}


// ---- spectrum of G = A_sigma^{-1} M (Section 2.4's figure): M = -alpha on PDE rows, +i k
// on EDGE rows (M^H: -alpha, -i k) ----

__device__ __forceinline__ bool an_corner(int i, int j, int n)
{
    return (i == 0 || i == n) && (j == 0 || j == n);
}

// block sum of three doubles into part[3 b + 0..2]
__device__ __forceinline__ void an_sum3(double a, double b, double c, double* __restrict__ part)
{
    __shared__ double sm[3][AN_NT / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
        c += __shfl_xor_sync(0xffffffffu, c, o);
    }
    if ((threadIdx.x & 31) == 0) {
        sm[0][threadIdx.x >> 5] = a;
        sm[1][threadIdx.x >> 5] = b;
        sm[2][threadIdx.x >> 5] = c;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double t = 0.0;
        for (int w = 0; w < AN_NT / 32; ++w) t += sm[threadIdx.x][w];
        part[3 * blockIdx.x + threadIdx.x] = t;
    }
}

// rhs = s M x in the inner precision (hole rows 0)
template <typename R>
__global__ void __launch_bounds__(AN_NT)
k_an_mx(const double2* __restrict__ x, const unsigned char* __restrict__ typ, typename CX<R>::T* __restrict__ rhs,
        long total, double s, double alpha, double k)
{
    typedef typename CX<R>::T c2;
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
        const unsigned char ty = typ[t];
        const double2 v = x[t];
        double rx = 0.0, ry = 0.0;
        if (ty == AN_PDE) {
            rx = -alpha * s * v.x;
            ry = -alpha * s * v.y;
        } else if (ty == AN_EDGE) {            // i k (v.x + i v.y)
            rx = -k * s * v.y;
            ry = k * s * v.x;
        }
        c2 r;
        r.x = an_narrow(rx, R());
        r.y = an_narrow(ry, R());
        rhs[t] = r;
    }
}

// power-iteration bookkeeping: sums of |e|^2 and of conj(x) e (re, im) per block, then x := e
template <typename R>
__global__ void __launch_bounds__(AN_NT)
k_an_pdot(double2* __restrict__ x, const typename CX<R>::T* __restrict__ e, const unsigned char* __restrict__ typ,
          long total, double* __restrict__ part)
{
    double a = 0.0, cr = 0.0, ci = 0.0;
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
        if (typ[t] == AN_HOLE) {
            x[t] = make_double2(0.0, 0.0);
            continue;
        }
        const double ex = an_widen(e[t].x), ey = an_widen(e[t].y);
        const double2 xv = x[t];
        a += ex * ex + ey * ey;
        cr += xv.x * ex + xv.y * ey;
        ci += xv.x * ey - xv.y * ex;
        x[t] = make_double2(ex, ey);
    }
    an_sum3(a, cr, ci, part);
}

// Adjoint solve, first half.  With W = 1 on PDE rows and -1/h on EDGE rows, W A_sigma is
// symmetric once the corner rows and columns are dropped, and no other row references a
// corner; so A^{-T} y is: corners h y_c; the rest W A^{-1} W^{-1} (y + the corner rows'
// transposed couplings, +y_c / 2 on each corner's two inward neighbours), the solve taken
// with zero right-hand side at the corners.  This kernel forms that right-hand side from
// y = e, writes the corners' part of z = M^H A^{-T} y (-i k h y_c) into x, and sums |y|^2.
template <typename R>
__global__ void __launch_bounds__(AN_NT)
k_an_tprep(const typename CX<R>::T* __restrict__ e, typename CX<R>::T* __restrict__ rhs, double2* __restrict__ x,
           const unsigned char* __restrict__ typ, int n, double h, double k, double* __restrict__ part)
{
    typedef typename CX<R>::T c2;
    const int S = n + 1;
    const long total = (long)S * S;
    double a = 0.0;
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
        const unsigned char ty = typ[t];
        c2 r;
        r.x = 0;
        r.y = 0;
        if (ty == AN_HOLE) {
            rhs[t] = r;
            x[t] = make_double2(0.0, 0.0);
            continue;
        }
        const int q = (int)t, i = q / S, j = q % S;
        double yx = an_widen(e[q].x), yy = an_widen(e[q].y);
        a += yx * yx + yy * yy;
        if (an_corner(i, j, n)) {
            rhs[q] = r;
            x[q] = make_double2(k * h * yy, -k * h * yx);     // -i k h y_c
            continue;
        }
        if (ty == AN_EDGE) {
            if ((j == 0 || j == n) && (i == 1 || i == n - 1)) {
                const c2 c = e[(i == 1 ? 0 : n) * S + j];
                yx += 0.5 * an_widen(c.x);
                yy += 0.5 * an_widen(c.y);
            }
            if ((i == 0 || i == n) && (j == 1 || j == n - 1)) {
                const c2 c = e[i * S + (j == 1 ? 0 : n)];
                yx += 0.5 * an_widen(c.x);
                yy += 0.5 * an_widen(c.y);
            }
            yx *= -h;
            yy *= -h;
        }
        r.x = an_narrow(yx, R());
        r.y = an_narrow(yy, R());
        rhs[q] = r;
    }
    an_sum3(a, 0.0, 0.0, part);
}

// Adjoint solve, second half: z = M^H W s off the corners (PDE: -alpha s; EDGE: (-i k) (-s / h)
// = (i k / h) s) into x; sums |z|^2 over every node (the corners' z from k_an_tprep)
template <typename R>
__global__ void __launch_bounds__(AN_NT)
k_an_tfin(const typename CX<R>::T* __restrict__ e, double2* __restrict__ x, const unsigned char* __restrict__ typ,
          int n, double h, double alpha, double k, double* __restrict__ part)
{
    const int S = n + 1;
    const long total = (long)S * S;
    double a = 0.0;
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
        const unsigned char ty = typ[t];
        if (ty == AN_HOLE) continue;
        const int q = (int)t, i = q / S, j = q % S;
        double2 z;
        if (an_corner(i, j, n)) {
            z = x[q];
        } else {
            const double sx = an_widen(e[q].x), sy = an_widen(e[q].y);
            if (ty == AN_PDE) {
                z.x = -alpha * sx;
                z.y = -alpha * sy;
            } else {
                z.x = -k / h * sy;
                z.y = k / h * sx;
            }
            x[q] = z;
        }
        a += z.x * z.x + z.y * z.y;
    }
    an_sum3(a, 0.0, 0.0, part);
}

// Lanczos on the real symmetric K = A^T D A, D = diag(1 / alpha^2 on PDE rows, 1 / k^2 on EDGE
// rows) = (G^{-1})^H G^{-1}: its largest eigenvalue is 1 / sigma_min(G)^2.  y = D A v:
__global__ void __launch_bounds__(AN_NT)
k_an_lz_a(const double* __restrict__ v, double* __restrict__ y, const unsigned char* __restrict__ typ, int n,
          double h, double sigma, double dp, double de)
{
    const int S = n + 1;
    const long total = (long)S * S;
    const double ih2 = 1.0 / (h * h), ih = 1.0 / h;
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
        const unsigned char ty = typ[t];
        const int q = (int)t, i = q / S, j = q % S;
        double r = 0.0;
        if (ty == AN_PDE) {
            // hole entries of v are zero
            r = (((v[q - S] + v[q + S]) + (v[q - 1] + v[q + 1])) - 4.0 * v[q]) * ih2 - sigma * v[q];
            r *= dp;
        } else if (ty == AN_EDGE) {
            double m = 0.0;
            int c = 0;
            if (i == 0) { m += v[S + j]; ++c; }
            if (i == n) { m += v[(n - 1) * S + j]; ++c; }
            if (j == 0) { m += v[i * S + 1]; ++c; }
            if (j == n) { m += v[i * S + n - 1]; ++c; }
            if (c == 2) m *= 0.5;
            r = (v[q] - m) * ih * de;
        }
        y[q] = r;
    }
}

// w = A^T y - beta v_prev (A^T gathered: PDE column j: its own row, its PDE neighbours'
// rows (1/h^2) and its EDGE neighbours' rows (-1/h, j being their inward neighbour); EDGE
// column: its own row (1/h), its inward neighbour's row (1/h^2), and the rows of the
// corners whose inward neighbour it is (-1/(2h)); corner column: its own row (1/h));
// part[3 b] = sum v . w
__global__ void __launch_bounds__(AN_NT)
k_an_lz_at(const double* __restrict__ y, const double* __restrict__ v, const double* __restrict__ vp, double beta,
           double* __restrict__ w, const unsigned char* __restrict__ typ, int n, double h, double sigma,
           double* __restrict__ part)
{
    const int S = n + 1;
    const long total = (long)S * S;
    const double ih2 = 1.0 / (h * h), ih = 1.0 / h;
    double a = 0.0;
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
        const unsigned char ty = typ[t];
        const int q = (int)t, i = q / S, j = q % S;
        double r = 0.0;
        if (ty == AN_PDE) {
            r = (-4.0 * ih2 - sigma) * y[q];
            const int nb[4] = {q - S, q + S, q - 1, q + 1};
#pragma unroll
            for (int d = 0; d < 4; ++d) {
                const unsigned char tn = typ[nb[d]];
                if (tn == AN_PDE) r += ih2 * y[nb[d]];
                else if (tn == AN_EDGE) r -= ih * y[nb[d]];
            }
        } else if (ty == AN_EDGE) {
            r = ih * y[q];
            if (!an_corner(i, j, n)) {
                const int in = (i == 0) ? S + j : (i == n) ? (n - 1) * S + j : (j == 0) ? i * S + 1 : i * S + n - 1;
                r += ih2 * y[in];
                if ((j == 0 || j == n) && (i == 1 || i == n - 1)) r -= 0.5 * ih * y[(i == 1 ? 0 : n) * S + j];
                if ((i == 0 || i == n) && (j == 1 || j == n - 1)) r -= 0.5 * ih * y[i * S + (j == 1 ? 0 : n)];
            }
        }
        r -= beta * vp[q];
        w[q] = r;
        a += v[q] * r;
    }
    an_sum3(a, 0.0, 0.0, part);
}

// w -= a v, part[3 b] = sum w^2
__global__ void __launch_bounds__(AN_NT)
k_an_lz_orth(double* __restrict__ w, const double* __restrict__ v, double a, long total, double* __restrict__ part)
{
    double s = 0.0;
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
        const double r = w[t] - a * v[t];
        w[t] = r;
        s += r * r;
    }
    an_sum3(s, 0.0, 0.0, part);
}

// v = s w; a seeded start vector when w == nullptr (hole nodes 0); part[3 b] = sum v^2
__global__ void __launch_bounds__(AN_NT)
k_an_lz_scale(double* __restrict__ v, const double* __restrict__ w, double s, const unsigned char* __restrict__ typ,
              long total, double* __restrict__ part)
{
    double a = 0.0;
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
        double r;
        if (w) {
            r = s * w[t];
        } else {
            unsigned long long z = 0x9e3779b97f4a7c15ull * (unsigned long long)(t + 1);
            z = (z ^ (z >> 31)) * 0xbf58476d1ce4e5b9ull;
            z ^= z >> 29;
            r = (typ[t] == AN_HOLE) ? 0.0 : ((double)(z >> 11) * (1.0 / 9007199254740992.0) - 0.5);
        }
        v[t] = r;
        a += r * r;
    }
    an_sum3(a, 0.0, 0.0, part);
}

// complex seeded start vector (hole 0) into x; part: sums of |x|^2
__global__ void __launch_bounds__(AN_NT)
k_an_seed(double2* __restrict__ x, const unsigned char* __restrict__ typ, long total, double* __restrict__ part)
{
    double a = 0.0;
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
        unsigned long long z = 0xd1b54a32d192ed03ull * (unsigned long long)(t + 7);
        z = (z ^ (z >> 31)) * 0xbf58476d1ce4e5b9ull;
        z ^= z >> 29;
        const double re = (double)(z >> 11) * (1.0 / 9007199254740992.0) - 0.5;
        z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
        z ^= z >> 31;
        const double im = (double)(z >> 11) * (1.0 / 9007199254740992.0) - 0.5;
        const double2 v = (typ[t] == AN_HOLE) ? make_double2(0.0, 0.0) : make_double2(re, im);
        x[t] = v;
        a += v.x * v.x + v.y * v.y;
    }
    an_sum3(a, 0.0, 0.0, part);
}

}  // namespace
}  // namespace helm

using namespace helm;

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct helm_annulus {
    int N = 0, prec = HELM_PREC_MIXED;
    double side = 1.0, hole = 0.15, k = 0.0, alpha = 0.0, sigma = 0.0;
    int nu1 = 2, nu2 = 2, cycles = 1;
    struct Level {
        int n;
        double h;
        unsigned char* typ;
        void* e;
        void* rhs;
        void* e2;                         // the swept iterate between the tile kernels
        int b0, b1, lo, hi;               // band ring [b0, b1]^2 minus the hole box [lo, hi]^2
        size_t band_bytes;                // shared memory of k_an_band_s (0: the L2 form)
    };
    std::vector<Level> lev;
    double* Ainv = nullptr;
    int* map = nullptr;
    int m = 0;
    double2* U1 = nullptr;
    double* part = nullptr;
    double* h_part = nullptr;
    int nblk = 0;
    unsigned long long* kmin = nullptr;
    cudaStream_t stream = nullptr;
    std::vector<void*> allocs;
    bool tiles = false;                   // the levels above the tail use the tile kernels
    cudaStream_t ls = nullptr;            // where an_vcycle and the step launch (stream, or cap)
    cudaStream_t cap = nullptr;           // non-blocking stream for capturing a step's graph
    bool capturing = false;
    uint64_t captured = 0;                // kernels recorded by the capture in progress
    int t0 = -1;                          // first level of the one-CTA coarse tail
    size_t tail_bytes = 0;
};

namespace {

#define AN_CK(call)                                                                             \
    do {                                                                                        \
        cudaError_t _e = (call);                                                                \
        if (_e != cudaSuccess) {                                                                \
            char _b[200];                                                                       \
            snprintf(_b, sizeof _b, "%s: %s", #call, cudaGetErrorString(_e));                   \
            note_error(_b);                                                                     \
            return HELM_ECUDA;                                                                  \
        }                                                                                       \
    } while (0)

// node types of a level (the oracle's rule: closed hole, outer edge rows elsewhere)
std::vector<unsigned char> an_types(int n, double side, double hole)
{
    const double h = side / n, eps = 1e-9 * side;
    std::vector<unsigned char> t((size_t)(n + 1) * (n + 1), AN_PDE);
    for (int i = 0; i <= n; ++i)
        for (int j = 0; j <= n; ++j) {
            const double x = -0.5 * side + i * h, y = -0.5 * side + j * h;
            unsigned char v = AN_PDE;
            if (i == 0 || i == n || j == 0 || j == n) v = AN_EDGE;
            if (std::fabs(x) <= hole + eps && std::fabs(y) <= hole + eps) v = AN_HOLE;
            t[(size_t)i * (n + 1) + j] = v;
        }
    return t;
}

bool an_geometry_ok(const std::vector<unsigned char>& t, int n)
{
    bool any = false;
    for (int i = 0; i <= n; ++i)
        for (int j = 0; j <= n; ++j) {
            const bool hole = t[(size_t)i * (n + 1) + j] == AN_HOLE;
            any |= hole;
            if (hole && (i <= 1 || i >= n - 1 || j <= 1 || j >= n - 1)) return false;
        }
    return any;
}

// dense inverse of the coarsest level's A_sigma on its unknowns (Gauss-Jordan, partial pivots)
bool an_coarse_inverse(const std::vector<unsigned char>& t, int n, double h, double sigma,
                       std::vector<double>& inv, std::vector<int>& map)
{
    const int S = n + 1;
    std::vector<int> idx((size_t)S * S, -1);
    map.clear();
    for (int q = 0; q < S * S; ++q)
        if (t[q] != AN_HOLE) { idx[q] = (int)map.size(); map.push_back(q); }
    const int m = (int)map.size();
    std::vector<double> A((size_t)m * m, 0.0);
    for (int r = 0; r < m; ++r) {
        const int q = map[r], i = q / S, j = q % S;
        if (t[q] == AN_PDE) {
            A[(size_t)r * m + r] = -4.0 / (h * h) - sigma;
            const int nb[4] = {q - S, q + S, q - 1, q + 1};
            for (int c : nb)
                if (idx[c] >= 0) A[(size_t)r * m + idx[c]] += 1.0 / (h * h);
        } else {
            std::vector<int> in;
            if (i == 0) in.push_back(q + S);
            if (i == n) in.push_back(q - S);
            if (j == 0) in.push_back(q + 1);
            if (j == n) in.push_back(q - 1);
            A[(size_t)r * m + r] = 1.0 / h;
            for (int c : in) A[(size_t)r * m + idx[c]] -= 1.0 / (h * in.size());
        }
    }
    inv.assign((size_t)m * m, 0.0);
    for (int r = 0; r < m; ++r) inv[(size_t)r * m + r] = 1.0;
    for (int c = 0; c < m; ++c) {
        int p = c;
        for (int r = c + 1; r < m; ++r)
            if (std::fabs(A[(size_t)r * m + c]) > std::fabs(A[(size_t)p * m + c])) p = r;
        if (std::fabs(A[(size_t)p * m + c]) < 1e-300) return false;
        if (p != c)
            for (int k = 0; k < m; ++k) {
                std::swap(A[(size_t)p * m + k], A[(size_t)c * m + k]);
                std::swap(inv[(size_t)p * m + k], inv[(size_t)c * m + k]);
            }
        const double d = A[(size_t)c * m + c];
        for (int k = 0; k < m; ++k) {
            A[(size_t)c * m + k] /= d;
            inv[(size_t)c * m + k] /= d;
        }
        for (int r = 0; r < m; ++r) {
            if (r == c) continue;
            const double f = A[(size_t)r * m + c];
            if (f == 0.0) continue;
            for (int k = 0; k < m; ++k) {
                A[(size_t)r * m + k] -= f * A[(size_t)c * m + k];
                inv[(size_t)r * m + k] -= f * inv[(size_t)c * m + k];
            }
        }
    }
    return true;
}

// kernels launched (or recorded into a step graph, counted at each replay)
void an_count(helm_annulus* a, uint64_t n)
{
    if (a->capturing) a->captured += n;
    else add_launches(n);
}

template <typename R>
helm_status an_vcycle(helm_annulus* a, int l, bool zero)
{
    typedef typename CX<R>::T c2;
    const auto& L = a->lev[l];
    cudaStream_t s = a->ls;
    if (l == a->t0) {                      // this level and all coarser ones in one CTA
        AnTail T{};
        T.L = (int)a->lev.size() - l;
        T.nu1 = a->nu1;
        T.nu2 = a->nu2;
        T.load_e = zero ? 0 : 1;
        T.m = a->m;
        T.sigma = a->sigma;
        T.Ainv = a->Ainv;
        T.map = a->map;
        for (int i = 0; i < T.L; ++i) {
            const auto& V = a->lev[l + i];
            T.lev[i] = AnTailLev{V.n, V.b0, V.b1, V.lo, V.hi, V.h, 1.0 / (4.0 + a->sigma * V.h * V.h), V.typ};
        }
        k_an_tail<R><<<1, 1024, a->tail_bytes, s>>>((c2*)L.e, (const c2*)L.rhs, T);
        AN_CK(cudaGetLastError());
        an_count(a, 1);
        return HELM_OK;
    }
    if (l + 1 == (int)a->lev.size()) {
        k_an_coarse<R><<<1, AN_NT, 0, s>>>((const c2*)L.rhs, (c2*)L.e, a->Ainv, a->map, a->m);
        AN_CK(cudaGetLastError());
        an_count(a, 1);
        return HELM_OK;
    }
    const R h = (R)L.h, dinv = (R)(1.0 / (4.0 + a->sigma * L.h * L.h));
    const int half = (L.n + 2) / 2;
    const int g = grid_for((long)(L.n + 1) * half);
    const auto& C = a->lev[l + 1];
    const bool tiles = a->tiles;
    // with the tile kernels the iterate goes e -> e2 (descent), e2 (correction, band),
    // e2 -> e (ascent)
    c2* const ew = (c2*)(tiles ? L.e2 : L.e);
    if (tiles) {
        const int ntc = (C.n + AN_CT) / AN_CT;
        k_an_down<R><<<ntc * ntc, AN_NT, an_down_bytes<R>(a->nu1), s>>>(
            (const c2*)L.e, ew, (const c2*)L.rhs, L.typ, L.n, h, dinv, (R)a->sigma, a->nu1, zero ? 0 : 1, (c2*)C.rhs,
            (c2*)C.e, C.typ, C.n);
        an_count(a, 1);
    } else {
        for (int sweep = 0; sweep < a->nu1; ++sweep)
            for (int col = 0; col < 2; ++col) {
                k_an_rbgs<R><<<g, AN_NT, 0, s>>>((c2*)L.e, (const c2*)L.rhs, L.typ, L.n, h, dinv, col, 0, L.n, 0,
                                                 L.n);
                an_count(a, 1);
            }
        k_an_restrict<R><<<grid_for((long)(C.n + 1) * (C.n + 1)), AN_NT, 0, s>>>(
            (const c2*)L.e, (const c2*)L.rhs, L.typ, L.n, h, (R)a->sigma, (c2*)C.rhs, (c2*)C.e, C.typ, C.n,
            (zero && a->nu1 == 0) ? 1 : 0);
        an_count(a, 1);
    }
    helm_status st = an_vcycle<R>(a, l + 1, true);
    if (st != HELM_OK) return st;
    k_an_prolong<R><<<grid_for((long)(L.n + 1) * (L.n + 1)), AN_NT, 0, s>>>((const c2*)C.e, C.n, ew, L.typ, L.n);
    if (L.band_bytes)
        k_an_band_s<R><<<1, 1024, L.band_bytes, s>>>(ew, (const c2*)L.rhs, L.typ, L.n, h, dinv,
                                                    AnRing(L.b0, L.b1, L.lo, L.hi), AN_BAND_SWEEPS);
    else
        k_an_band<R><<<1, 1024, 0, s>>>(ew, (const c2*)L.rhs, L.typ, L.n, h, dinv, L.b0, L.b1, L.lo, L.hi,
                                        AN_BAND_SWEEPS);
    an_count(a, 2);
    if (tiles) {                           // nu2 = 0: the launch only moves e2 to e
        const int nt = (L.n + AN_FT) / AN_FT;
        k_an_up<R><<<nt * nt, AN_NT, an_win_bytes<R>(an_up_sw(a->nu2)), s>>>(ew, (c2*)L.e, (const c2*)L.rhs,
                                                                            L.typ, L.n, h, dinv, a->nu2);
        an_count(a, 1);
    } else {
        for (int sweep = 0; sweep < a->nu2; ++sweep)
            for (int col = 0; col < 2; ++col) {
                k_an_rbgs<R><<<g, AN_NT, 0, s>>>((c2*)L.e, (const c2*)L.rhs, L.typ, L.n, h, dinv, col, 0, L.n, 0,
                                                 L.n);
                an_count(a, 1);
            }
    }
    AN_CK(cudaGetLastError());
    return HELM_OK;
}

template <typename R>
helm_status an_solve(helm_annulus* a, const double2* data, double2* u, double tol, int max_outer, int* iters,
                     double* hist, int* final_status)
{
    typedef typename CX<R>::T c2;
    cudaStream_t s = a->stream;
    a->ls = s;
    const auto& L0 = a->lev[0];
    const long total = (long)(a->N + 1) * (a->N + 1);
    double2* U[2] = {u, a->U1};
    k_an_init<<<grid_for(total), AN_NT, 0, s>>>(U[0], U[1], data, L0.typ, total);
    add_launches(1);
    // mode 0: the start residual; mode 1: an outer step's update and residual; both end
    // with the norm partials copied to the host (the caller synchronises)
    auto enqueue = [&](int mode, int it) -> helm_status {
        cudaStream_t q = a->ls;
        if (mode == 1) {
            for (int c = 0; c < a->cycles; ++c) {
                if (c == 0) AN_CK(cudaMemsetAsync(L0.e, 0, total * sizeof(c2), q));
                const helm_status st = an_vcycle<R>(a, 0, c == 0);
                if (st != HELM_OK) return st;
            }
            k_an_update<R><<<a->nblk, AN_NT, 0, q>>>(U[(it - 1) & 1], U[it & 1], (const c2*)L0.e, L0.typ, total,
                                                     a->part);
            an_count(a, 1);
        }
        k_an_resid<R><<<a->nblk, AN_NT, 0, q>>>(U[mode == 1 ? (it & 1) : 0], data, L0.typ, (c2*)L0.rhs, a->N,
                                                L0.h, a->k * a->k, a->k, a->part);
        an_count(a, 1);
        AN_CK(cudaGetLastError());
        AN_CK(cudaMemcpyAsync(a->h_part, a->part, 2 * sizeof(double) * a->nblk, cudaMemcpyDeviceToHost, q));
        return HELM_OK;
    };
    // an outer step of either parity as one graph (its pointers and parameters are fixed for
    // this solve); without graphs the step's launches are issued one by one
    cudaGraphExec_t gx[2] = {nullptr, nullptr};
    uint64_t gn[2] = {0, 0};
    auto drop_graphs = [&]() {
        for (int p = 0; p < 2; ++p)
            if (gx[p]) cudaGraphExecDestroy(gx[p]);
    };
    if (AN_GRAPHS && max_outer > 0) {
        for (int p = 0; p < 2; ++p) {
            cudaGraph_t gr = nullptr;
            if (cudaStreamBeginCapture(a->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) break;
            a->ls = a->cap;
            a->capturing = true;
            a->captured = 0;
            const helm_status est = enqueue(1, p == 1 ? 1 : 2);
            a->capturing = false;
            a->ls = s;
            const cudaError_t ce = cudaStreamEndCapture(a->cap, &gr);
            if (est != HELM_OK || ce != cudaSuccess || !gr ||
                cudaGraphInstantiate(&gx[p], gr, 0) != cudaSuccess) {
                if (gr) cudaGraphDestroy(gr);
                gx[p] = nullptr;
                break;
            }
            cudaGraphDestroy(gr);
            gn[p] = a->captured;
        }
        if (!gx[0] || !gx[1]) {                // no graphs: launch step by step
            drop_graphs();
            gx[0] = gx[1] = nullptr;
            cudaGetLastError();
        }
    }
    auto step = [&](int mode, int it) -> helm_status {
        if (mode == 1 && gx[0]) {
            AN_CK(cudaGraphLaunch(gx[it & 1], s));
            add_launches(gn[it & 1]);
        } else {
            const helm_status st = enqueue(mode, it);
            if (st != HELM_OK) return st;
        }
        AN_CK(cudaStreamSynchronize(s));
        return HELM_OK;
    };
    // start: r_0 = b from U[0] (the hole data, zero elsewhere)
    helm_status st = step(0, 1);
    if (st != HELM_OK) { drop_graphs(); return st; }
    double r2 = 0.0;
    for (int b = 0; b < a->nblk; ++b) r2 += a->h_part[2 * b];
    const double norm0 = std::sqrt(r2);
    int it = 0, status = HELM_MAXITER, run = 0;
    double prev = 1.0, rmin = 1.0;
    if (hist) hist[0] = (norm0 == 0.0) ? 0.0 : 1.0;
    if (norm0 == 0.0 || !std::isfinite(norm0)) status = std::isfinite(norm0) ? HELM_CONVERGED : HELM_ENONFINITE;
    else {
        for (it = 1; it <= max_outer; ++it) {
            st = step(1, it);
            if (st != HELM_OK) { drop_graphs(); return st; }
            r2 = 0.0;
            for (int b = 0; b < a->nblk; ++b) r2 += a->h_part[2 * b];
            const double rel = std::sqrt(r2) / norm0;
            if (hist) hist[it] = rel;
            // the cavity's status rule
            if (!std::isfinite(rel)) { status = HELM_ENONFINITE; break; }
            if (rel <= tol) { status = HELM_CONVERGED; break; }
            if (rel > 1e4) { status = HELM_DIVERGED; break; }
            run = (rel >= prev) ? run + 1 : 0;
            prev = rel;
            rmin = std::min(rmin, rel);
            if (it >= 20 && run >= 10 && rel >= 2.0 * rmin) { status = HELM_DIVERGED; break; }
        }
        if (it > max_outer) it = max_outer;
    }
    drop_graphs();
    // the result lives in U[it & 1]: the caller's buffer is U[0]
    if (it & 1) AN_CK(cudaMemcpyAsync(u, a->U1, total * sizeof(double2), cudaMemcpyDeviceToDevice, s));
    AN_CK(cudaStreamSynchronize(s));
    if (iters) *iters = it;
    *final_status = status;
    return HELM_OK;
}


// ---- spectrum of G (Section 2.4's figure) ----

// e := A_sigma^{-1} rhs on level 0 by `cycles` multigrid cycles from zero
template <typename R>
helm_status an_apply_inv(helm_annulus* a, int cycles)
{
    typedef typename CX<R>::T c2;
    const auto& L0 = a->lev[0];
    const long total = (long)(a->N + 1) * (a->N + 1);
    a->ls = a->stream;
    for (int c = 0; c < cycles; ++c) {
        if (c == 0) AN_CK(cudaMemsetAsync(L0.e, 0, total * sizeof(c2), a->stream));
        const helm_status st = an_vcycle<R>(a, 0, c == 0);
        if (st != HELM_OK) return st;
    }
    return HELM_OK;
}

// per-call reduction buffers (three doubles per block) and their host copy
struct AnSums {
    double* d = nullptr;
    double* h = nullptr;
    int nb = 0;
    ~AnSums()
    {
        if (d) cudaFree(d);
        if (h) cudaFreeHost(h);
    }
    helm_status init(int nblk)
    {
        nb = nblk;
        if (cudaMalloc(&d, 3 * sizeof(double) * nb) != cudaSuccess) return HELM_ENOMEM;
        if (cudaMallocHost(&h, 3 * sizeof(double) * nb) != cudaSuccess) return HELM_ENOMEM;
        return HELM_OK;
    }
    // block sums -> out[0..2] (fixed order)
    helm_status fetch(cudaStream_t s, double* out)
    {
        AN_CK(cudaMemcpyAsync(h, d, 3 * sizeof(double) * nb, cudaMemcpyDeviceToHost, s));
        AN_CK(cudaStreamSynchronize(s));
        out[0] = out[1] = out[2] = 0.0;
        for (int b = 0; b < nb; ++b)
            for (int c = 0; c < 3; ++c) out[c] += h[3 * b + c];
        return HELM_OK;
    }
};

// Power iteration x <- G x / ||G x||: rho ~ ||G x|| (||x|| = 1), lambda ~ x^H G x.
template <typename R>
helm_status an_spectral(helm_annulus* a, int max_iter, double tol, int cycles, double* rho, double* lre,
                        double* lim, int* iters, bool* conv)
{
    typedef typename CX<R>::T c2;
    const auto& L0 = a->lev[0];
    const long total = (long)(a->N + 1) * (a->N + 1);
    cudaStream_t s = a->stream;
    AnSums sums;
    helm_status st = sums.init(a->nblk);
    if (st != HELM_OK) return st;
    double v[3];
    k_an_seed<<<a->nblk, AN_NT, 0, s>>>(a->U1, L0.typ, total, sums.d);
    an_count(a, 1);
    if ((st = sums.fetch(s, v)) != HELM_OK) return st;
    double sc = 1.0 / std::sqrt(v[0]), prev = 0.0, r = 0.0;
    int ok = 0, it = 0;
    *conv = false;
    for (it = 1; it <= max_iter; ++it) {
        k_an_mx<R><<<a->nblk, AN_NT, 0, s>>>(a->U1, L0.typ, (c2*)L0.rhs, total, sc, a->alpha, a->k);
        an_count(a, 1);
        if ((st = an_apply_inv<R>(a, cycles)) != HELM_OK) return st;
        k_an_pdot<R><<<a->nblk, AN_NT, 0, s>>>(a->U1, (const c2*)L0.e, L0.typ, total, sums.d);
        an_count(a, 1);
        AN_CK(cudaGetLastError());
        if ((st = sums.fetch(s, v)) != HELM_OK) return st;
        r = std::sqrt(v[0]);
        *lre = sc * v[1];
        *lim = sc * v[2];
        if (!(r > 0.0) || !std::isfinite(r)) return HELM_ENONFINITE;
        sc = 1.0 / r;
        ok = (std::fabs(r - prev) <= tol * r) ? ok + 1 : 0;
        prev = r;
        if (ok >= 2) {
            *conv = true;
            break;
        }
    }
    *rho = r;
    *iters = std::min(it, max_iter);
    return HELM_OK;
}

// largest eigenvalue of the symmetric tridiagonal matrix (diag a[0..m-1], off-diagonal
// b[1..m-1]) by bisection on the Sturm count
double tridiag_max(const std::vector<double>& a, const std::vector<double>& b, int m)
{
    double lo = 1e300, hi = -1e300;
    for (int i = 0; i < m; ++i) {
        const double r = (i > 0 ? std::fabs(b[i]) : 0.0) + (i + 1 < m ? std::fabs(b[i + 1]) : 0.0);
        lo = std::min(lo, a[i] - r);
        hi = std::max(hi, a[i] + r);
    }
    auto below = [&](double x) {                  // eigenvalues < x
        int c = 0;
        double d = 1.0;
        for (int i = 0; i < m; ++i) {
            d = a[i] - x - (i > 0 ? b[i] * b[i] / d : 0.0);
            if (d == 0.0) d = -1e-300;
            if (d < 0.0) ++c;
        }
        return c;
    };
    for (int k = 0; k < 200 && hi - lo > 1e-15 * std::max(std::fabs(lo), std::fabs(hi)); ++k) {
        const double mid = 0.5 * (lo + hi);
        if (below(mid) >= m) hi = mid;
        else lo = mid;
    }
    return 0.5 * (lo + hi);
}

// sigma_max(G) by power iteration on G^H G (adjoint solves through the symmetrised
// operator), sigma_min(G) = 1 / sqrt(lambda_max(A^T D A)) by Lanczos (no solves).
template <typename R>
helm_status an_singular(helm_annulus* a, int max_iter, double tol, int cycles, double* smax, double* smin,
                        int* iters, bool* conv)
{
    typedef typename CX<R>::T c2;
    const auto& L0 = a->lev[0];
    const int n = a->N;
    const long total = (long)(n + 1) * (n + 1);
    cudaStream_t s = a->stream;
    AnSums sums;
    helm_status st = sums.init(a->nblk);
    if (st != HELM_OK) return st;
    double v[3];
    // sigma_max
    k_an_seed<<<a->nblk, AN_NT, 0, s>>>(a->U1, L0.typ, total, sums.d);
    an_count(a, 1);
    if ((st = sums.fetch(s, v)) != HELM_OK) return st;
    double sc = 1.0 / std::sqrt(v[0]), prev = 0.0, est = 0.0;
    int ok = 0, it1 = 0;
    bool c1 = false;
    for (it1 = 1; it1 <= max_iter; ++it1) {
        k_an_mx<R><<<a->nblk, AN_NT, 0, s>>>(a->U1, L0.typ, (c2*)L0.rhs, total, sc, a->alpha, a->k);
        an_count(a, 1);
        if ((st = an_apply_inv<R>(a, cycles)) != HELM_OK) return st;
        k_an_tprep<R><<<a->nblk, AN_NT, 0, s>>>((const c2*)L0.e, (c2*)L0.rhs, a->U1, L0.typ, n, L0.h, a->k, sums.d);
        an_count(a, 1);
        if ((st = sums.fetch(s, v)) != HELM_OK) return st;
        est = std::sqrt(v[0]);
        if ((st = an_apply_inv<R>(a, cycles)) != HELM_OK) return st;
        k_an_tfin<R><<<a->nblk, AN_NT, 0, s>>>((const c2*)L0.e, a->U1, L0.typ, n, L0.h, a->alpha, a->k, sums.d);
        an_count(a, 1);
        AN_CK(cudaGetLastError());
        if ((st = sums.fetch(s, v)) != HELM_OK) return st;
        if (!(v[0] > 0.0) || !std::isfinite(v[0])) return HELM_ENONFINITE;
        sc = 1.0 / std::sqrt(v[0]);
        ok = (std::fabs(est - prev) <= tol * est) ? ok + 1 : 0;
        prev = est;
        if (ok >= 2) {
            c1 = true;
            break;
        }
    }
    *smax = est;
    // sigma_min: Lanczos on the real K = A^T D A
    double* buf = nullptr;
    if (cudaMalloc(&buf, 4 * total * sizeof(double)) != cudaSuccess) return HELM_ENOMEM;
    struct Free {
        double* p;
        ~Free() { cudaFree(p); }
    } fr{buf};
    double *vp = buf, *vc = buf + total, *w = buf + 2 * total, *y = buf + 3 * total;
    AN_CK(cudaMemsetAsync(vp, 0, total * sizeof(double), s));
    k_an_lz_scale<<<a->nblk, AN_NT, 0, s>>>(vc, nullptr, 0.0, L0.typ, total, sums.d);
    if ((st = sums.fetch(s, v)) != HELM_OK) return st;
    k_an_lz_scale<<<a->nblk, AN_NT, 0, s>>>(vc, vc, 1.0 / std::sqrt(v[0]), L0.typ, total, sums.d);
    an_count(a, 2);
    const double dp = 1.0 / (a->alpha * a->alpha), de = 1.0 / (a->k * a->k);
    std::vector<double> al, be(1, 0.0);
    double beta = 0.0, theta = 0.0, tprev = 0.0;
    int it2 = 0;
    bool c2ok = false;
    ok = 0;
    for (it2 = 1; it2 <= max_iter; ++it2) {
        k_an_lz_a<<<a->nblk, AN_NT, 0, s>>>(vc, y, L0.typ, n, L0.h, a->sigma, dp, de);
        k_an_lz_at<<<a->nblk, AN_NT, 0, s>>>(y, vc, vp, beta, w, L0.typ, n, L0.h, a->sigma, sums.d);
        an_count(a, 2);
        if ((st = sums.fetch(s, v)) != HELM_OK) return st;
        const double alpha = v[0];
        k_an_lz_orth<<<a->nblk, AN_NT, 0, s>>>(w, vc, alpha, total, sums.d);
        an_count(a, 1);
        AN_CK(cudaGetLastError());
        if ((st = sums.fetch(s, v)) != HELM_OK) return st;
        al.push_back(alpha);
        beta = std::sqrt(v[0]);
        theta = tridiag_max(al, be, (int)al.size());
        be.push_back(beta);
        ok = (std::fabs(theta - tprev) <= tol * theta) ? ok + 1 : 0;
        tprev = theta;
        if (ok >= 2 || !(beta > 1e-300 * theta)) {
            c2ok = true;
            break;
        }
        // v_prev <- v, v <- w / beta (into the old v_prev buffer)
        k_an_lz_scale<<<a->nblk, AN_NT, 0, s>>>(vp, w, 1.0 / beta, L0.typ, total, sums.d);
        an_count(a, 1);
        std::swap(vp, vc);
    }
    AN_CK(cudaStreamSynchronize(s));
    if (!(theta > 0.0) || !std::isfinite(theta)) return HELM_ENONFINITE;
    *smin = 1.0 / std::sqrt(theta);
    *iters = std::max(std::min(it1, max_iter), std::min(it2, max_iter));
    *conv = c1 && c2ok;
    return HELM_OK;
}

}  // namespace

extern "C" {

helm_status helm_annulus_create(helm_annulus** out, int n, double side, double hole, double k, int prec)
{
    if (!out) return HELM_EINVAL;
    *out = nullptr;
    if (n < 16 || n > 16384 || (n & (n - 1))) return HELM_EINVAL;
    if (!(side > 0.0) || !std::isfinite(side) || !(hole > 0.0) || !(hole < 0.5 * side)) return HELM_EINVAL;
    if (!(k >= 0.0) || !std::isfinite(k) || (prec != HELM_PREC_FP64 && prec != HELM_PREC_MIXED)) return HELM_EINVAL;
    helm_annulus* a = new helm_annulus();
    a->N = n;
    a->side = side;
    a->hole = hole;
    a->k = k;
    a->alpha = k * k;
    a->sigma = 0.0;
    a->prec = prec;
    auto fail = [&](helm_status st) { helm_annulus_destroy(a); return st; };
    // a blocking stream: its work is ordered after the caller's work on the legacy default
    // stream (where the inputs were written)
    if (cudaStreamCreate(&a->stream) != cudaSuccess) return fail(HELM_ECUDA);
    if (cudaStreamCreateWithFlags(&a->cap, cudaStreamNonBlocking) != cudaSuccess) return fail(HELM_ECUDA);
    a->ls = a->stream;
    const size_t eb = prec == HELM_PREC_FP64 ? 16 : 8;
    for (int m = n; m >= AN_NC; m /= 2) {
        std::vector<unsigned char> t = an_types(m, side, hole);
        if (!an_geometry_ok(t, m)) return fail(HELM_EINVAL);
        helm_annulus::Level L{};
        L.n = m;
        L.h = side / m;
        const size_t pts = (size_t)(m + 1) * (m + 1);
        void* p = nullptr;
        const size_t pb = ((pts * eb + 255) / 256) * 256;
        if (cudaMalloc(&p, ((pts + 255) / 256) * 256 + 3 * pb) != cudaSuccess) return fail(HELM_ENOMEM);
        a->allocs.push_back(p);
        L.typ = (unsigned char*)p;
        L.e = (char*)p + ((pts + 255) / 256) * 256;
        L.rhs = (char*)L.e + pb;
        L.e2 = (char*)L.rhs + pb;
        if (cudaMemcpy(L.typ, t.data(), pts, cudaMemcpyHostToDevice) != cudaSuccess) return fail(HELM_ECUDA);
        if (cudaMemset(L.e, 0, pts * eb) != cudaSuccess || cudaMemset(L.rhs, 0, pts * eb) != cudaSuccess ||
            cudaMemset(L.e2, 0, pts * eb) != cudaSuccess)
            return fail(HELM_ECUDA);
        // band: the hole's index box [lo, hi]^2 (centred square) widened by AN_BAND nodes
        int lo = m, hi = 0;
        for (int i = 0; i <= m; ++i)
            if (t[(size_t)i * (m + 1) + m / 2] == AN_HOLE) { lo = std::min(lo, i); hi = std::max(hi, i); }
        L.lo = lo;
        L.hi = hi;
        L.b0 = std::max(1, lo - AN_BAND);
        L.b1 = std::min(m - 1, hi + AN_BAND);
        L.band_bytes = 0;
        if (AN_BAND_SMEM) {
            const AnRing g(L.b0, L.b1, L.lo, L.hi);
            const size_t bb = prec == HELM_PREC_FP64 ? an_band_bytes<double>(g) : an_band_bytes<float>(g);
            if (bb <= AN_SMEM_MAX && g.total() <= 1024 * AN_BAND_PT) L.band_bytes = bb;
        }
        a->lev.push_back(L);
    }
    if (a->lev.size() < 2) return fail(HELM_EINVAL);
    // the coarse tail: levels of at most `top` intervals (at most AN_TAIL_MAX of them)
    const int top = prec == HELM_PREC_FP64 ? AN_TAIL_TOP_D : AN_TAIL_TOP_F;
    for (int l = 0; l < (int)a->lev.size(); ++l)
        if (a->lev[l].n <= top) { a->t0 = l; break; }
    if (a->t0 >= 0 && (int)a->lev.size() - a->t0 <= AN_TAIL_MAX) {
        int ns[AN_TAIL_MAX];
        const int L = (int)a->lev.size() - a->t0;
        for (int i = 0; i < L; ++i) ns[i] = a->lev[a->t0 + i].n;
        a->tail_bytes = (prec == HELM_PREC_FP64) ? an_tail_bytes<double>(ns, L) : an_tail_bytes<float>(ns, L);
        const cudaError_t e = (prec == HELM_PREC_FP64)
            ? cudaFuncSetAttribute(k_an_tail<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)a->tail_bytes)
            : cudaFuncSetAttribute(k_an_tail<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)a->tail_bytes);
        if (e != cudaSuccess) a->t0 = -1;      // no tail: per-level launches all the way down
        cudaGetLastError();
    } else {
        a->t0 = -1;
    }
    {
        const size_t dmax = (prec == HELM_PREC_FP64) ? an_down_bytes<double>(8) : an_down_bytes<float>(8);
        const size_t umax = (prec == HELM_PREC_FP64) ? an_win_bytes<double>(an_up_sw(8)) : an_win_bytes<float>(an_up_sw(8));
        cudaError_t e1, e2;
        if (prec == HELM_PREC_FP64) {
            e1 = cudaFuncSetAttribute(k_an_down<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dmax);
            e2 = cudaFuncSetAttribute(k_an_up<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)umax);
        } else {
            e1 = cudaFuncSetAttribute(k_an_down<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dmax);
            e2 = cudaFuncSetAttribute(k_an_up<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)umax);
        }
        if (e1 != cudaSuccess || e2 != cudaSuccess) return fail(HELM_ECUDA);
        // in FP64 the windows' redundant halo sweeps cost more than the launches they save
        a->tiles = AN_TILES && prec == HELM_PREC_MIXED;
    }
    size_t band_max = 0;
    for (const auto& L : a->lev) band_max = std::max(band_max, L.band_bytes);
    if (band_max) {
        const cudaError_t e = (prec == HELM_PREC_FP64)
            ? cudaFuncSetAttribute(k_an_band_s<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)band_max)
            : cudaFuncSetAttribute(k_an_band_s<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)band_max);
        if (e != cudaSuccess) return fail(HELM_ECUDA);
    }
    const long total = (long)(n + 1) * (n + 1);
    a->nblk = grid_for(total);
    void* p = nullptr;
    if (cudaMalloc(&p, total * sizeof(double2) + 2 * sizeof(double) * a->nblk + 256) != cudaSuccess)
        return fail(HELM_ENOMEM);
    a->allocs.push_back(p);
    a->U1 = (double2*)p;
    a->part = (double*)((char*)p + total * sizeof(double2));
    a->kmin = (unsigned long long*)((char*)a->part + 2 * sizeof(double) * a->nblk);
    if (cudaMallocHost(&a->h_part, 2 * sizeof(double) * a->nblk) != cudaSuccess) return fail(HELM_ENOMEM);
    helm_status st = helm_annulus_set_shift(a, a->alpha);
    if (st != HELM_OK) return fail(st);
    *out = a;
    return HELM_OK;
}

helm_status helm_annulus_destroy(helm_annulus* a)
{
    if (!a) return HELM_EINVAL;
    if (a->stream) cudaStreamSynchronize(a->stream);
    for (void* p : a->allocs) cudaFree(p);
    if (a->Ainv) cudaFree(a->Ainv);
    if (a->h_part) cudaFreeHost(a->h_part);
    if (a->stream) cudaStreamDestroy(a->stream);
    if (a->cap) cudaStreamDestroy(a->cap);
    delete a;
    return HELM_OK;
}

helm_status helm_annulus_set_shift(helm_annulus* a, double alpha)
{
    if (!a || !std::isfinite(alpha) || alpha < a->k * a->k) return HELM_EINVAL;
    a->alpha = alpha;
    a->sigma = (alpha == a->k * a->k) ? 0.0 : alpha - a->k * a->k;
    const auto& C = a->lev.back();
    std::vector<unsigned char> t = an_types(C.n, a->side, a->hole);
    std::vector<double> inv;
    std::vector<int> map;
    if (!an_coarse_inverse(t, C.n, C.h, a->sigma, inv, map)) return HELM_EINVAL;
    if (a->Ainv) cudaFree(a->Ainv);
    a->Ainv = nullptr;
    a->m = (int)map.size();
    void* p = nullptr;
    if (cudaMalloc(&p, inv.size() * sizeof(double) + map.size() * sizeof(int)) != cudaSuccess) return HELM_ENOMEM;
    a->Ainv = (double*)p;
    a->map = (int*)(a->Ainv + inv.size());
    AN_CK(cudaMemcpy(a->Ainv, inv.data(), inv.size() * sizeof(double), cudaMemcpyHostToDevice));
    AN_CK(cudaMemcpy(a->map, map.data(), map.size() * sizeof(int), cudaMemcpyHostToDevice));
    return HELM_OK;
}

helm_status helm_annulus_set_cycle(helm_annulus* a, int nu1, int nu2, int cycles)
{
    if (!a || nu1 < 0 || nu1 > 8 || nu2 < 0 || nu2 > 8 || nu1 + nu2 < 1 || cycles < 1 || cycles > 16)
        return HELM_EINVAL;
    a->nu1 = nu1;
    a->nu2 = nu2;
    a->cycles = cycles;
    return HELM_OK;
}

helm_status helm_annulus_solve(helm_annulus* a, const void* data, void* u, double tol, int max_outer, int* iters,
                               double* res_hist)
{
    if (!a || !(tol >= 0.0) || max_outer < 0) return HELM_EINVAL;
    if (!device_pointer_ok(data) || !device_pointer_ok(u) || data == u) return HELM_EINVAL;
    int status = HELM_MAXITER;
    const helm_status st = (a->prec == HELM_PREC_FP64)
        ? an_solve<double>(a, (const double2*)data, (double2*)u, tol, max_outer, iters, res_hist, &status)
        : an_solve<float>(a, (const double2*)data, (double2*)u, tol, max_outer, iters, res_hist, &status);
    return st != HELM_OK ? st : (helm_status)status;
}

helm_status helm_annulus_exit_times(helm_annulus* a, double c_tau, double tol, int max_outer, void* E_out,
                                    void* L_out, double* kstar)
{
    if (!a || !(c_tau > 0.0) || !std::isfinite(c_tau) || !(tol >= 0.0) || max_outer < 1) return HELM_EINVAL;
    if (!device_pointer_ok(E_out) || !device_pointer_ok(L_out) || E_out == L_out) return HELM_EINVAL;
    // Delta E = -c_tau, dE/dn = 0 and Delta L = 0, dL/dn = 1 (zero on the hole): the outer
    // iteration with k = 0 and no shift, i.e. FP64-refined multigrid solves of A_0
    helm_annulus* z = nullptr;
    helm_status st = helm_annulus_create(&z, a->N, a->side, a->hole, 0.0, a->prec);
    if (st != HELM_OK) return st;
    helm_annulus_set_cycle(z, a->nu1, a->nu2, a->cycles);
    const long total = (long)(a->N + 1) * (a->N + 1);
    std::vector<unsigned char> t = an_types(a->N, a->side, a->hole);
    std::vector<double2> hd(total);
    void* buf = nullptr;
    if (cudaMalloc(&buf, 2 * total * sizeof(double2)) != cudaSuccess) {
        helm_annulus_destroy(z);
        return HELM_ENOMEM;
    }
    double2* dd = (double2*)buf;
    double2* U = dd + total;
    auto done = [&](helm_status s) {
        cudaFree(buf);
        helm_annulus_destroy(z);
        return s;
    };
    for (int which = 0; which < 2; ++which) {
        for (long q = 0; q < total; ++q)
            hd[q] = make_double2(t[q] == AN_PDE ? (which == 0 ? -c_tau : 0.0) : (t[q] == AN_EDGE && which == 1 ? 1.0 : 0.0),
                                 0.0);
        if (cudaMemcpy(dd, hd.data(), total * sizeof(double2), cudaMemcpyHostToDevice) != cudaSuccess)
            return done(HELM_ECUDA);
        int it = 0;
        st = helm_annulus_solve(z, dd, U, tol, max_outer, &it, nullptr);
        if (st != HELM_CONVERGED) return done(st < 0 ? st : HELM_MAXITER);
        k_an_real<<<grid_for(total), AN_NT, 0, z->stream>>>(U, (double*)(which == 0 ? E_out : L_out), total);
        add_launches(1);
    }
    if (kstar) {
        const unsigned long long init = 0x7ff0000000000000ull;      // +inf
        if (cudaMemcpyAsync(z->kmin, &init, sizeof init, cudaMemcpyHostToDevice, z->stream) != cudaSuccess)
            return done(HELM_ECUDA);
        k_an_kstar<<<grid_for(total), AN_NT, 0, z->stream>>>((const double*)E_out, (const double*)L_out,
                                                             z->lev[0].typ, total, z->kmin);
        add_launches(1);
        unsigned long long bits = 0;
        if (cudaMemcpyAsync(&bits, z->kmin, sizeof bits, cudaMemcpyDeviceToHost, z->stream) != cudaSuccess ||
            cudaStreamSynchronize(z->stream) != cudaSuccess)
            return done(HELM_ECUDA);
        double v;
        memcpy(&v, &bits, sizeof v);
        *kstar = v;
    }
    if (cudaStreamSynchronize(z->stream) != cudaSuccess) return done(HELM_ECUDA);
    return done(HELM_OK);
}

helm_status helm_annulus_spectral_radius(helm_annulus* a, int max_iters, double tol, int cycles, double* rho,
                                         double* lambda_re, double* lambda_im, int* iters_done)
{
    if (!a || max_iters < 1 || !(tol > 0.0) || cycles < 1 || cycles > 64) return HELM_EINVAL;
    double r = 0.0, lr = 0.0, li = 0.0;
    int it = 0;
    bool conv = false;
    const helm_status st = (a->prec == HELM_PREC_FP64)
        ? an_spectral<double>(a, max_iters, tol, cycles, &r, &lr, &li, &it, &conv)
        : an_spectral<float>(a, max_iters, tol, cycles, &r, &lr, &li, &it, &conv);
    if (st != HELM_OK) return st;
    if (rho) *rho = r;
    if (lambda_re) *lambda_re = lr;
    if (lambda_im) *lambda_im = li;
    if (iters_done) *iters_done = it;
    return conv ? HELM_OK : HELM_MAXITER;
}

helm_status helm_annulus_condition(helm_annulus* a, int max_iters, double tol, int cycles, double* sigma_max,
                                   double* sigma_min, double* cond, int* iters_done)
{
    if (!a || max_iters < 1 || !(tol > 0.0) || cycles < 1 || cycles > 64 || !(a->k > 0.0)) return HELM_EINVAL;
    double smax = 0.0, smin = 0.0;
    int it = 0;
    bool conv = false;
    const helm_status st = (a->prec == HELM_PREC_FP64)
        ? an_singular<double>(a, max_iters, tol, cycles, &smax, &smin, &it, &conv)
        : an_singular<float>(a, max_iters, tol, cycles, &smax, &smin, &it, &conv);
    if (st != HELM_OK) return st;
    if (sigma_max) *sigma_max = smax;
    if (sigma_min) *sigma_min = smin;
    if (cond) *cond = smax / smin;
    if (iters_done) *iters_done = it;
    return conv ? HELM_OK : HELM_MAXITER;
}

}  // extern "C"
