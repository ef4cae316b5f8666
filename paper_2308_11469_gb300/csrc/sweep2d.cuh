// Colour-plane tiles and the red-black half-sweep of the fused 2D multigrid kernels
// (vcycle2d.cu), shared with the fused ascent + residual kernel (outer.cu).  half_sweep's
// warps stride over rows: NWARP = the CTA's warps (SW_NW for the 512-thread kernels).
#pragma once
#include "launch.h"

namespace helm {
namespace {

constexpr int SW_NT = 512;
constexpr int SW_NW = SW_NT / 32;

template <typename T> __device__ __forceinline__ T cz() { T v; v.x = 0; v.y = 0; return v; }

// Shared-memory tiles are stored as two colour planes: node (lx, ly) of the staged
// window, whose global colour is (gx + gy) & 1, lives in plane[colour] at row ly, column
// lx >> 1 (row stride W/2).  A warp that updates 32 nodes of one colour in a row then
// reads its west / east / north / south neighbours (the other colour) and its own rhs as
// contiguous runs: no shared-memory bank conflicts.
template <int W>
struct Planes {
    static constexpr int WH = W / 2;
    __device__ __forceinline__ static int at(int lx, int ly) { return ly * WH + (lx >> 1); }
};

// One half-sweep over the nodes of colour `color` within Chebyshev distance `ring` of
// the tile, clipped to the interior.  E0/E1, R0/R1: colour planes of the window whose
// element (0, 0) is global node (gx0, gy0).
template <typename R, int W, int TX, int TY, int NWARP = SW_NW>
__device__ __forceinline__ void half_sweep(typename C2<R>::T* E0, typename C2<R>::T* E1,
                                           const typename C2<R>::T* R0,
                                           const typename C2<R>::T* R1, int gx0, int gy0,
                                           int x0, int y0, int ring, int n, R h2, R dinv, int color)
{
    typedef typename C2<R>::T c2;
    typedef Planes<W> PL;
    const int xa = max(x0 - ring, 1), xb = min(x0 + TX - 1 + ring, n);
    const int ya = max(y0 - ring, 1), yb = min(y0 + TY - 1 + ring, n);
    const int lane = threadIdx.x & 31;
    c2* __restrict__ Ec = color ? E1 : E0;
    const c2* __restrict__ Eo = color ? E0 : E1;
    const c2* __restrict__ Rc = color ? R1 : R0;
    for (int gy = ya + (int)(threadIdx.x >> 5); gy <= yb; gy += NWARP) {
        const int xs = xa + (((xa + gy) & 1) ^ color);
        const int ly = gy - gy0;
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int gx = xs + 2 * (lane + 32 * j);
            if (gx > xb) break;
            const int lx = gx - gx0;
            const int o = PL::at(lx, ly);
            const c2 a = Eo[PL::at(lx - 1, ly)], b = Eo[PL::at(lx + 1, ly)];
            const c2 c = Eo[PL::at(lx, ly - 1)], d = Eo[PL::at(lx, ly + 1)];
            const c2 rr = Rc[o];
            c2 v;
            v.x = ((a.x + b.x + c.x + d.x) - h2 * rr.x) * dinv;
            v.y = ((a.y + b.y + c.y + d.y) - h2 * rr.y) * dinv;
            Ec[o] = v;
        }
    }
}

}  // namespace
}  // namespace helm
