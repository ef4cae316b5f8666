// Fused 2D multigrid kernels: two launches per level and V-cycle.
//
//   k_down2d  pre-smoothing (nu1 red-black sweeps) + residual + full-weighting
//             restriction, on a 64 x 32 tile staged in shared memory with a halo of
//             2 nu1 + 2 nodes.  Each red (then black) half-sweep updates a region one
//             node narrower than the previous one, so after the nu1 sweeps the
//             iterate is exact on the tile plus a 2-node ring, the residual on the tile
//             plus a 1-node ring, and the restriction of every coarse node owned by
//             the tile (fine index 2I inside the tile) needs nothing from other tiles.
//             The halo values are recomputed from the same inputs by every tile that
//             needs them, so they equal the owner's values bit for bit.
//             Reads the iterate (or treats it as zero) and rhs; writes the smoothed
//             iterate to the level's second buffer e2 and the coarse rhs.
//   k_up2d    prolongation + correction + post-smoothing (nu2 sweeps): loads e2 on the
//             tile plus a 2 nu2 ring, adds the multilinear interpolation of the coarse
//             level's final iterate, smooths in shared memory, writes the tile to e.
// Reading one buffer and writing the other keeps tiles free of read/write races.
//
// The node colours, the update formula and the transfer weights are those of the
// generic kernels (vcycle.cu), so both paths compute the same V-cycle.
#include "launch.h"

namespace helm {
namespace {

constexpr int TX = 64;
constexpr int TY = 32;
constexpr int NT = 256;

template <typename T> __device__ __forceinline__ T cz() { T v; v.x = 0; v.y = 0; return v; }

__device__ __forceinline__ size_t goff(const LevelDesc& L, int x, int y) {
    return (size_t)y * (size_t)L.pitch + x;
}

// One half-sweep over the nodes of colour `color` whose distance to the tile is at
// most `ring` (Chebyshev), restricted to interior nodes.  E, Rh: shared arrays with
// row stride W, origin (gx0, gy0) = global coordinates of shared element (0, 0).
template <typename R>
__device__ __forceinline__ void half_sweep(typename C2<R>::T* E, const typename C2<R>::T* Rh,
                                           int W, int Hh, int gx0, int gy0, int x0, int y0,
                                           int ring, int n, R h2, int color)
{
    typedef typename C2<R>::T c2;
    const R inv = (R)0.25;
    // region in global coordinates, clipped to the interior
    const int xa = max(x0 - ring, 1), xb = min(x0 + TX - 1 + ring, n);
    const int ya = max(y0 - ring, 1), yb = min(y0 + TY - 1 + ring, n);
    const int w = xb - xa + 1;
    if (w <= 0 || yb < ya) return;
    // pairs along x: the node of this colour in {x, x+1}
    const int pw = (w + 1) >> 1;
    const int total = pw * (yb - ya + 1);
    for (int q = threadIdx.x; q < total; q += NT) {
        const int gy = ya + q / pw;
        int gx = xa + 2 * (q % pw);
        if (((gx + gy) & 1) != color) ++gx;
        if (gx > xb) continue;
        const int o = (gy - gy0) * W + (gx - gx0);
        const c2 a = E[o - 1], b = E[o + 1], c = E[o - W], d = E[o + W];
        const c2 rr = Rh[o];
        c2 v;
        v.x = ((a.x + b.x + c.x + d.x) - h2 * rr.x) * inv;
        v.y = ((a.y + b.y + c.y + d.y) - h2 * rr.y) * inv;
        E[o] = v;
    }
}

template <typename R>
__global__ void __launch_bounds__(NT)
k_down2d(const InstDesc* __restrict__ insts, const InstState* __restrict__ st,
         const MgItem* __restrict__ items, int nu1, int zero_mode)
{
    typedef typename C2<R>::T c2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const MgItem item = items[blockIdx.y];
    if (st[item.inst].status != HELM_ST_ACTIVE) return;
    const LevelDesc L = insts[item.inst].lev[item.level];
    const LevelDesc C = insts[item.inst].lev[item.level + 1];
    const int n = L.n;
    const int ntx = (n + TX - 1) / TX;
    const int nty = (n + TY - 1) / TY;
    if ((int)blockIdx.x >= ntx * nty) return;
    const int x0 = 1 + (blockIdx.x % ntx) * TX;
    const int y0 = 1 + (blockIdx.x / ntx) * TY;
    const int H = 2 * nu1 + 2;
    const int W = TX + 2 * H, Hh = TY + 2 * H;
    c2* E = reinterpret_cast<c2*>(smem_raw);
    c2* Rs = E + W * Hh;
    const int gx0 = x0 - H, gy0 = y0 - H;
    const bool zero = (zero_mode == 2) || (zero_mode == 1 && item.level > 0);
    const c2* ge = (const c2*)L.e;
    const c2* gr = (const c2*)L.rhs;
    // stage e (zero outside the padded grid, or everywhere when known zero) and rhs
    for (int q = threadIdx.x; q < W * Hh; q += NT) {
        const int gx = gx0 + q % W, gy = gy0 + q / W;
        const bool in = gx >= 1 && gx <= n && gy >= 1 && gy <= n;
        E[q] = (!zero && in) ? ge[goff(L, gx, gy)] : cz<c2>();
        Rs[q] = in ? gr[goff(L, gx, gy)] : cz<c2>();
    }
    __syncthreads();
    const R h2 = (R)(L.h * L.h);
    int ring = 2 * nu1 + 1;
    for (int s = 0; s < nu1; ++s) {
        half_sweep<R>(E, Rs, W, Hh, gx0, gy0, x0, y0, ring--, n, h2, 0);
        __syncthreads();
        half_sweep<R>(E, Rs, W, Hh, gx0, gy0, x0, y0, ring--, n, h2, 1);
        __syncthreads();
    }
    // smoothed iterate of the tile -> e2
    c2* ge2 = (c2*)L.e2;
    for (int q = threadIdx.x; q < TX * TY; q += NT) {
        const int gx = x0 + q % TX, gy = y0 + q / TX;
        if (gx <= n && gy <= n) ge2[goff(L, gx, gy)] = E[(gy - gy0) * W + (gx - gx0)];
    }
    // residual on the tile plus a 1-node ring, in place of rhs
    const R ih2 = (R)1 / h2;
    {
        const int xa = max(x0 - 1, 1), xb = min(x0 + TX, n);
        const int ya = max(y0 - 1, 1), yb = min(y0 + TY, n);
        const int w = xb - xa + 1;
        const int total = w * (yb - ya + 1);
        for (int q = threadIdx.x; q < total; q += NT) {
            const int gx = xa + q % w, gy = ya + q / w;
            const int o = (gy - gy0) * W + (gx - gx0);
            const c2 c = E[o], a = E[o - 1], b = E[o + 1], u = E[o - W], d = E[o + W];
            const c2 rr = Rs[o];
            c2 v;
            v.x = rr.x - ((a.x + b.x + u.x + d.x) - (R)4 * c.x) * ih2;
            v.y = rr.y - ((a.y + b.y + u.y + d.y) - (R)4 * c.y) * ih2;
            Rs[o] = v;
        }
    }
    __syncthreads();
    // full weighting at the coarse nodes owned by this tile
    c2* cr = (c2*)C.rhs;
    const int nc = C.n;
    const int Xa = (x0 + 1) >> 1, Xb = min((x0 + TX - 1) >> 1, nc);
    const int Ya = (y0 + 1) >> 1, Yb = min((y0 + TY - 1) >> 1, nc);
    const int cw = Xb - Xa + 1;
    if (cw > 0 && Yb >= Ya) {
        const int total = cw * (Yb - Ya + 1);
        for (int q = threadIdx.x; q < total; q += NT) {
            const int X = Xa + q % cw, Y = Ya + q / cw;
            const int o = (2 * Y - gy0) * W + (2 * X - gx0);
            R ax = 0, ay = 0;
#pragma unroll
            for (int dy = -1; dy <= 1; ++dy) {
                const R wy = (dy == 0) ? (R)2 : (R)1;
#pragma unroll
                for (int dx = -1; dx <= 1; ++dx) {
                    const R wgt = wy * ((dx == 0) ? (R)2 : (R)1);
                    const c2 r = Rs[o + dy * W + dx];
                    ax += wgt * r.x;
                    ay += wgt * r.y;
                }
            }
            c2 v;
            v.x = ax * (R)(1.0 / 16.0);
            v.y = ay * (R)(1.0 / 16.0);
            cr[goff(C, X, Y)] = v;
        }
    }
}

template <typename R>
__global__ void __launch_bounds__(NT)
k_up2d(const InstDesc* __restrict__ insts, const InstState* __restrict__ st,
       const MgItem* __restrict__ items, int nu2)
{
    typedef typename C2<R>::T c2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const MgItem item = items[blockIdx.y];
    if (st[item.inst].status != HELM_ST_ACTIVE) return;
    const LevelDesc L = insts[item.inst].lev[item.level];
    const LevelDesc C = insts[item.inst].lev[item.level + 1];
    const int n = L.n;
    const int ntx = (n + TX - 1) / TX;
    const int nty = (n + TY - 1) / TY;
    if ((int)blockIdx.x >= ntx * nty) return;
    const int x0 = 1 + (blockIdx.x % ntx) * TX;
    const int y0 = 1 + (blockIdx.x / ntx) * TY;
    const int H = 2 * nu2;
    const int W = TX + 2 * H, Hh = TY + 2 * H;
    c2* E = reinterpret_cast<c2*>(smem_raw);
    c2* Rs = E + W * Hh;
    c2* Cs = Rs + W * Hh;
    const int gx0 = x0 - H, gy0 = y0 - H;
    // coarse window covering the region: X in [cx0, cx0 + CW)
    const int cx0 = max(gx0, 0) >> 1, cy0 = max(gy0, 0) >> 1;
    const int cx1 = min((gx0 + W) >> 1, C.n + 1), cy1 = min((gy0 + Hh) >> 1, C.n + 1);
    const int CW = cx1 - cx0 + 1, CH = cy1 - cy0 + 1;
    const c2* gce = (const c2*)C.e;
    for (int q = threadIdx.x; q < CW * CH; q += NT) {
        const int X = cx0 + q % CW, Y = cy0 + q / CW;
        Cs[q] = gce[goff(C, X, Y)];
    }
    const c2* ge2 = (const c2*)L.e2;
    const c2* gr = (const c2*)L.rhs;
    __syncthreads();
    for (int q = threadIdx.x; q < W * Hh; q += NT) {
        const int gx = gx0 + q % W, gy = gy0 + q / W;
        const bool in = gx >= 1 && gx <= n && gy >= 1 && gy <= n;
        c2 v = cz<c2>();
        c2 r = cz<c2>();
        if (in) {
            v = ge2[goff(L, gx, gy)];
            r = gr[goff(L, gx, gy)];
            const int X0 = (gx >> 1) - cx0, X1 = ((gx + 1) >> 1) - cx0;
            const int Y0 = (gy >> 1) - cy0, Y1 = ((gy + 1) >> 1) - cy0;
            const c2 a = Cs[Y0 * CW + X0], b = Cs[Y0 * CW + X1];
            const c2 c = Cs[Y1 * CW + X0], d = Cs[Y1 * CW + X1];
            v.x += (R)0.25 * (((a.x + b.x) + c.x) + d.x);
            v.y += (R)0.25 * (((a.y + b.y) + c.y) + d.y);
        }
        E[q] = v;
        Rs[q] = r;
    }
    __syncthreads();
    const R h2 = (R)(L.h * L.h);
    int ring = 2 * nu2 - 1;
    for (int s = 0; s < nu2; ++s) {
        half_sweep<R>(E, Rs, W, Hh, gx0, gy0, x0, y0, ring--, n, h2, 0);
        __syncthreads();
        half_sweep<R>(E, Rs, W, Hh, gx0, gy0, x0, y0, ring--, n, h2, 1);
        __syncthreads();
    }
    c2* ge = (c2*)L.e;
    for (int q = threadIdx.x; q < TX * TY; q += NT) {
        const int gx = x0 + q % TX, gy = y0 + q / TX;
        if (gx <= n && gy <= n) ge[goff(L, gx, gy)] = E[(gy - gy0) * W + (gx - gx0)];
    }
}

}  // namespace

size_t down2d_smem(int prec, int nu1)
{
    const int H = 2 * nu1 + 2;
    return (size_t)2 * (TX + 2 * H) * (TY + 2 * H) * (prec == 0 ? 16 : 8);
}

size_t up2d_smem(int prec, int nu2)
{
    const int H = 2 * nu2;
    const int W = TX + 2 * H, Hh = TY + 2 * H;
    const int CW = W / 2 + 2, CH = Hh / 2 + 2;
    return ((size_t)2 * W * Hh + (size_t)CW * CH) * (prec == 0 ? 16 : 8);
}

int tiles2d(int n) { return ((n + TX - 1) / TX) * ((n + TY - 1) / TY); }

template <typename R>
static cudaError_t attrs2d()
{
    const int prec = sizeof(R) == 8 ? 0 : 1;
    cudaError_t e = cudaFuncSetAttribute(k_down2d<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)down2d_smem(prec, 8));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_up2d<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)up2d_smem(prec, 8));
}

cudaError_t setup_2d(int prec) { return prec == 0 ? attrs2d<double>() : attrs2d<float>(); }

cudaError_t launch_down2d(int prec, const InstDesc* insts, const InstState* st, const MgItem* items,
                          int nitems, int max_tiles, int nu1, int zero_mode, cudaStream_t s)
{
    dim3 g(max_tiles, nitems);
    const size_t sm = down2d_smem(prec, nu1);
    if (prec == 0) k_down2d<double><<<g, NT, sm, s>>>(insts, st, items, nu1, zero_mode);
    else k_down2d<float><<<g, NT, sm, s>>>(insts, st, items, nu1, zero_mode);
    return cudaGetLastError();
}

cudaError_t launch_up2d(int prec, const InstDesc* insts, const InstState* st, const MgItem* items,
                        int nitems, int max_tiles, int nu2, cudaStream_t s)
{
    dim3 g(max_tiles, nitems);
    const size_t sm = up2d_smem(prec, nu2);
    if (prec == 0) k_up2d<double><<<g, NT, sm, s>>>(insts, st, items, nu2);
    else k_up2d<float><<<g, NT, sm, s>>>(insts, st, items, nu2);
    return cudaGetLastError();
}

}  // namespace helm
