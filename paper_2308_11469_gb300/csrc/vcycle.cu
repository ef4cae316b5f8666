// Geometric-multigrid kernels for the inner problem (Delta_h - sigma) e = rhs, e = 0 on
// the wall: every outer step of the paper's iteration (Section 2.2, Eq. (2.6);
// sigma = alpha - k^2, 0 for alpha = k^2) is one such real problem per real/imaginary
// lane.  The paper prescribes no inner solver; this file is the library's choice (see
// the header).  sigma enters the local solve (diagonal 2D/h^2 + sigma) and the residual.
//
// Generic (any D in {2, 3}, float or double) kernels over lists of (instance, level)
// work items, blocks striding over each item's nodes:
//   k_rbgs      red-black Gauss-Seidel half-sweep (node colour = parity of the sum of
//               its padded indices; red = 0); each updated node solves its own equation.
//   k_restrict  coarse rhs = full weighting ([1,2,1]/4 per axis) of the fine residual
//               rhs - Delta_h e, coarse iterate = 0.
//   k_prolong   e_fine += multilinear interpolation of e_coarse.
// The coarse levels (n <= 63 in 2D, n <= 15 in 3D) run inside one CTA (tail.cu).
#include "launch.h"
#include "pdl.cuh"

namespace helm {
namespace {

template <int D>
__device__ __forceinline__ size_t rowoff(const LevelDesc& L, int y, int z) {
    return ((D == 3) ? ((size_t)z * L.rows + y) : (size_t)y) * (size_t)L.pitch;
}
template <int D>
__device__ __forceinline__ size_t off(const LevelDesc& L, int x, int y, int z) {
    return rowoff<D>(L, y, z) + xslot<D>(x, L.pitch);
}

template <typename T> __device__ __forceinline__ T cz() { T v; v.x = 0; v.y = 0; return v; }

// ---------------------------------------------------------------------------
// Red-black Gauss-Seidel half-sweep
// ---------------------------------------------------------------------------
template <int D, typename R>
__global__ void __launch_bounds__(256)
k_rbgs(const InstDesc* __restrict__ insts, const InstState* __restrict__ st,
       const MgItem* __restrict__ items, int color, int mode)
{
    pdl_wait();
    pdl_trigger();
    typedef typename C2<R>::T c2;
    const MgItem item = items[blockIdx.y];
    const InstState sv = st[item.inst];
    if (sv.status != HELM_ST_ACTIVE) return;
    const LevelDesc L = insts[item.inst].lev[item.level];
    const int n = L.n, half = (n + 1) >> 1;
    const int rows = (D == 3) ? n * n : n;
    c2* __restrict__ e = (c2*)L.e;
    const c2* __restrict__ r = (const c2*)lev_rhs(L, item.level, sv.it);
    const long P = L.pitch;
    const long PL = (long)L.pitch * L.rows;
    const R h2 = (R)(L.h * L.h);
    const R inv = (R)L.dinv;                       // 1 / (2D + sigma h^2)
    // mode 2: the iterate of every level is zero; mode 1: only levels > 0 are (their
    // iterate was cleared by the restriction); mode 0: plain half-sweep.
    const bool zi = (mode == 2) || (mode == 1 && item.level > 0);
    // a warp per grid row (y, z), its lanes over the row's node pairs
    const int wpb = blockDim.x >> 5, lane = threadIdx.x & 31;
    for (int row = blockIdx.x * wpb + (threadIdx.x >> 5); row < rows; row += gridDim.x * wpb) {
      const int y = (D == 3) ? row % n + 1 : row + 1;
      const int z = (D == 3) ? row / n + 1 : 0;
      for (int j = lane; j < half; j += 32) {
        const int xa = 2 * j + 1;                       // pair {xa, xa + 1}
        const int xc = (((xa + y + z) & 1) == color) ? xa : xa + 1;
        const int xo = (xc == xa) ? xa + 1 : xa;
        if (xc <= n) {
            const long rb = (long)rowoff<D>(L, y, z);
            const long o = rb + xslot<D>(xc, L.pitch);
            const c2 rr = r[o];
            c2 v;
            if (zi) {                                   // all neighbours are zero
                v.x = -h2 * rr.x * inv;
                v.y = -h2 * rr.y * inv;
            } else {
                const c2 a = e[rb + xslot<D>(xc - 1, L.pitch)], b = e[rb + xslot<D>(xc + 1, L.pitch)];
                const c2 c = e[o - P], d = e[o + P];
                R sx = a.x + b.x + c.x + d.x;
                R sy = a.y + b.y + c.y + d.y;
                if (D == 3) {
                    const c2 f = e[o - PL], g = e[o + PL];
                    sx += f.x + g.x;
                    sy += f.y + g.y;
                }
                v.x = (sx - h2 * rr.x) * inv;
                v.y = (sy - h2 * rr.y) * inv;
            }
            e[o] = v;
        }
        if (zi && xo <= n) e[off<D>(L, xo, y, z)] = cz<c2>();
      }
    }
}

// ---------------------------------------------------------------------------
// Residual + full-weighting restriction
// ---------------------------------------------------------------------------
// mode 2 / 1: the fine iterate is zero on every level / on levels > 0 (no pre-smoothing
// from a zero iterate): the residual is rhs itself (the same values the general form gives
// with e = 0) and the coarse iterate is left for the prolongation to assign.
template <int D, typename R>
__global__ void __launch_bounds__(256)
k_restrict(const InstDesc* __restrict__ insts, const InstState* __restrict__ st,
           const MgItem* __restrict__ items, int mode)
{
    pdl_wait();
    pdl_trigger();
    typedef typename C2<R>::T c2;
    const MgItem item = items[blockIdx.y];
    const InstState sv = st[item.inst];
    if (sv.status != HELM_ST_ACTIVE) return;
    const LevelDesc F = insts[item.inst].lev[item.level];
    const LevelDesc C = insts[item.inst].lev[item.level + 1];
    const int nc = C.n;
    const int crows = (D == 3) ? nc * nc : nc;
    const c2* __restrict__ e = (const c2*)F.e;
    const c2* __restrict__ r = (const c2*)lev_rhs(F, item.level, sv.it);
    c2* __restrict__ cr = (c2*)C.rhs;
    c2* __restrict__ ce = (c2*)C.e;
    const long P = F.pitch;
    const long PL = (long)F.pitch * F.rows;
    const R ih2 = (R)(1.0 / (F.h * F.h));
    const R sig = (R)insts[item.inst].sigma;
    const R scale = (D == 3) ? (R)(1.0 / 64.0) : (R)(1.0 / 16.0);
    const bool ez = (mode == 2) || (mode == 1 && item.level > 0);
    // a warp per coarse row (Y, Z), its lanes over X
    const int wpb = blockDim.x >> 5, lane = threadIdx.x & 31;
    for (int row = blockIdx.x * wpb + (threadIdx.x >> 5); row < crows; row += gridDim.x * wpb) {
      const int Y = (D == 3) ? row % nc + 1 : row + 1;
      const int Z = (D == 3) ? row / nc + 1 : 0;
      for (int X = lane + 1; X <= nc; X += 32) {
        R ax = 0, ay = 0;
        const int zlo = (D == 3) ? -1 : 0, zhi = (D == 3) ? 1 : 0;
        if (ez) {
            for (int dz = zlo; dz <= zhi; ++dz) {
                const R wz = (D == 3) ? (dz == 0 ? (R)2 : (R)1) : (R)1;
                for (int dy = -1; dy <= 1; ++dy) {
                    const R wy = (dy == 0) ? (R)2 : (R)1;
                    for (int dx = -1; dx <= 1; ++dx) {
                        const R w = wz * wy * ((dx == 0) ? (R)2 : (R)1);
                        const c2 rr = r[(long)off<D>(F, 2 * X + dx, 2 * Y + dy, 2 * Z + dz)];
                        ax += w * rr.x;
                        ay += w * rr.y;
                    }
                }
            }
            const size_t oc = off<D>(C, X, Y, Z);
            c2 v;
            v.x = ax * scale;
            v.y = ay * scale;
            cr[oc] = v;
            continue;
        }
        for (int dz = zlo; dz <= zhi; ++dz) {
            const R wz = (D == 3) ? (dz == 0 ? (R)2 : (R)1) : (R)1;
            for (int dy = -1; dy <= 1; ++dy) {
                const R wy = (dy == 0) ? (R)2 : (R)1;
                for (int dx = -1; dx <= 1; ++dx) {
                    const R w = wz * wy * ((dx == 0) ? (R)2 : (R)1);
                    const long rb = (long)rowoff<D>(F, 2 * Y + dy, 2 * Z + dz);
                    const int x = 2 * X + dx;
                    const long o = rb + xslot<D>(x, F.pitch);
                    const c2 c = e[o], a = e[rb + xslot<D>(x - 1, F.pitch)], b = e[rb + xslot<D>(x + 1, F.pitch)];
                    const c2 u = e[o - P], d = e[o + P];
                    R sx = a.x + b.x + u.x + d.x;
                    R sy = a.y + b.y + u.y + d.y;
                    if (D == 3) {
                        const c2 f = e[o - PL], g = e[o + PL];
                        sx += f.x + g.x;
                        sy += f.y + g.y;
                    }
                    const c2 rr = r[o];
                    ax += w * ((rr.x - (sx - (R)(2 * D) * c.x) * ih2) + sig * c.x);
                    ay += w * ((rr.y - (sy - (R)(2 * D) * c.y) * ih2) + sig * c.y);
                }
            }
        }
        const size_t oc = off<D>(C, X, Y, Z);
        c2 v;
        v.x = ax * scale;
        v.y = ay * scale;
        cr[oc] = v;
        ce[oc] = cz<c2>();
      }
    }
}

// ---------------------------------------------------------------------------
// Multilinear prolongation + correction
// ---------------------------------------------------------------------------
// mode 2 / 1: the fine iterate is zero on every level / on levels > 0 (no pre-smoothing
// from a zero iterate): e := interpolation instead of e += interpolation.
template <int D, typename R>
__global__ void __launch_bounds__(256)
k_prolong(const InstDesc* __restrict__ insts, const InstState* __restrict__ st,
          const MgItem* __restrict__ items, int mode)
{
    pdl_wait();
    pdl_trigger();
    typedef typename C2<R>::T c2;
    const MgItem item = items[blockIdx.y];
    if (st[item.inst].status != HELM_ST_ACTIVE) return;
    const LevelDesc F = insts[item.inst].lev[item.level];
    const LevelDesc C = insts[item.inst].lev[item.level + 1];
    const int n = F.n;
    const int rows = (D == 3) ? n * n : n;
    c2* __restrict__ e = (c2*)F.e;
    const c2* __restrict__ ce = (const c2*)C.e;
    const bool ez = (mode == 2) || (mode == 1 && item.level > 0);
    // a warp per fine row (y, z), its lanes over x
    const int wpb = blockDim.x >> 5, lane = threadIdx.x & 31;
    for (int row = blockIdx.x * wpb + (threadIdx.x >> 5); row < rows; row += gridDim.x * wpb) {
      const int y = (D == 3) ? row % n + 1 : row + 1;
      const int z = (D == 3) ? row / n + 1 : 0;
      // a lane forms the fine pair x = 2p + 1 (coarse columns p, p + 1) and x = 2p + 2
      // (column p + 1 twice) from the same eight coarse values; per axis an even fine
      // index takes one coarse node (weight 1), an odd one two (1/2 each)
      const int y0 = y >> 1, y1 = (y + 1) >> 1;
      const int z0 = z >> 1, z1 = (z + 1) >> 1;
      const R w = (D == 3) ? (R)0.125 : (R)0.25;
      for (int p = lane; 2 * p + 1 <= n; p += 32) {
        c2 cv[2][2][2];                                 // [iz][iy][column p / p + 1]
        const int nz = (D == 3) ? 2 : 1;
#pragma unroll
        for (int iz = 0; iz < nz; ++iz)
#pragma unroll
            for (int iy = 0; iy < 2; ++iy) {
                const size_t rc = rowoff<D>(C, iy ? y1 : y0, iz ? z1 : z0);
                cv[iz][iy][0] = ce[rc + xslot<D>(p, C.pitch)];
                cv[iz][iy][1] = ce[rc + xslot<D>(p + 1, C.pitch)];
            }
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            const int x = 2 * p + 1 + half;
            if (x > n) break;
            // each of the 2^D corner reads counts 1/2^D; coincident corners (even index)
            // are read twice, which gives the weight 1 of an even fine index
            R vx = 0, vy = 0;
#pragma unroll
            for (int iz = 0; iz < nz; ++iz)
#pragma unroll
                for (int iy = 0; iy < 2; ++iy)
#pragma unroll
                    for (int ix = 0; ix < 2; ++ix) {
                        const c2 c = cv[iz][iy][half ? 1 : ix];
                        vx += c.x;
                        vy += c.y;
                    }
            const long o = (long)off<D>(F, x, y, z);
            c2 v;
            if (ez) {
                v.x = w * vx;
                v.y = w * vy;
            } else {
                v = e[o];
                v.x += w * vx;
                v.y += w * vy;
            }
            e[o] = v;
        }
      }
    }
}

template <int D, typename R>
__global__ void __launch_bounds__(256)
k_zero(const InstDesc* __restrict__ insts, const InstState* __restrict__ st,
       const MgItem* __restrict__ items)
{
    pdl_wait();
    pdl_trigger();
    typedef typename C2<R>::T c2;
    const MgItem item = items[blockIdx.y];
    if (st[item.inst].status != HELM_ST_ACTIVE) return;
    const LevelDesc L = insts[item.inst].lev[item.level];
    const long total = (D == 3) ? (long)L.pitch * L.rows * L.rows : (long)L.pitch * L.rows;
    c2* __restrict__ e = (c2*)L.e;
    for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < total;
         q += (long)gridDim.x * blockDim.x)
        e[q] = cz<c2>();
}

inline dim3 mg_grid(int work, int nitems) {
    int bx = (work + 255) / 256;
    if (bx < 1) bx = 1;
    if (bx > 1216) bx = 1216;   // 152 SMs x 8 blocks; blocks stride over larger levels
    return dim3(bx, nitems);
}

}  // namespace

template <int D, typename R>
static cudaError_t carve()
{
    cudaError_t e;
    if ((e = max_carveout(k_rbgs<D, R>)) != cudaSuccess) return e;
    if ((e = max_carveout(k_restrict<D, R>)) != cudaSuccess) return e;
    if ((e = max_carveout(k_prolong<D, R>)) != cudaSuccess) return e;
    return max_carveout(k_zero<D, R>);
}

cudaError_t setup_generic(int D, int prec)
{
    if (D == 2) return prec == 0 ? carve<2, double>() : carve<2, float>();
    return prec == 0 ? carve<3, double>() : carve<3, float>();
}

cudaError_t launch_rbgs(int D, int prec, const InstDesc* insts, const InstState* st,
                        const MgItem* items, int nitems, int work, int color, int mode,
                        cudaStream_t s)
{
    dim3 g = mg_grid(work, nitems);
    if (D == 2 && prec == 0) launch_k(k_rbgs<2, double>, dim3(g), dim3(256), 0, s, insts, st, items, color, mode);
    else if (D == 2) launch_k(k_rbgs<2, float>, dim3(g), dim3(256), 0, s, insts, st, items, color, mode);
    else if (prec == 0) launch_k(k_rbgs<3, double>, dim3(g), dim3(256), 0, s, insts, st, items, color, mode);
    else launch_k(k_rbgs<3, float>, dim3(g), dim3(256), 0, s, insts, st, items, color, mode);
    return cudaGetLastError();
}

cudaError_t launch_restrict(int D, int prec, const InstDesc* insts, const InstState* st,
                            const MgItem* items, int nitems, int work, cudaStream_t s, int mode)
{
    dim3 g = mg_grid(work, nitems);
    if (D == 2 && prec == 0) launch_k(k_restrict<2, double>, dim3(g), dim3(256), 0, s, insts, st, items, mode);
    else if (D == 2) launch_k(k_restrict<2, float>, dim3(g), dim3(256), 0, s, insts, st, items, mode);
    else if (prec == 0) launch_k(k_restrict<3, double>, dim3(g), dim3(256), 0, s, insts, st, items, mode);
    else launch_k(k_restrict<3, float>, dim3(g), dim3(256), 0, s, insts, st, items, mode);
    return cudaGetLastError();
}

cudaError_t launch_prolong(int D, int prec, const InstDesc* insts, const InstState* st,
                           const MgItem* items, int nitems, int work, cudaStream_t s, int mode)
{
    dim3 g = mg_grid(work, nitems);
    if (D == 2 && prec == 0) launch_k(k_prolong<2, double>, dim3(g), dim3(256), 0, s, insts, st, items, mode);
    else if (D == 2) launch_k(k_prolong<2, float>, dim3(g), dim3(256), 0, s, insts, st, items, mode);
    else if (prec == 0) launch_k(k_prolong<3, double>, dim3(g), dim3(256), 0, s, insts, st, items, mode);
    else launch_k(k_prolong<3, float>, dim3(g), dim3(256), 0, s, insts, st, items, mode);
    return cudaGetLastError();
}

cudaError_t launch_zero(int D, int prec, const InstDesc* insts, const InstState* st,
                        const MgItem* items, int nitems, int work, cudaStream_t s)
{
    dim3 g = mg_grid(work, nitems);
    if (D == 2 && prec == 0) launch_k(k_zero<2, double>, dim3(g), dim3(256), 0, s, insts, st, items);
    else if (D == 2) launch_k(k_zero<2, float>, dim3(g), dim3(256), 0, s, insts, st, items);
    else if (prec == 0) launch_k(k_zero<3, double>, dim3(g), dim3(256), 0, s, insts, st, items);
    else launch_k(k_zero<3, float>, dim3(g), dim3(256), 0, s, insts, st, items);
    return cudaGetLastError();
}

}  // namespace helm
