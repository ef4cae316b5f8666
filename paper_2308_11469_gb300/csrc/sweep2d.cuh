// Colour-plane tiles and the red-black half-sweep of the fused 2D multigrid kernels
// (vcycle2d.cu), shared with the fused ascent + residual kernel (outer.cu).
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

// One half-sweep over the nodes of colour COLOR within Chebyshev distance RING of the
// TX x TY tile at (x0, y0), clipped to the interior.  E0/E1, R0/R1: colour planes of the
// window whose element (0, 0) is global node (gx0, gy0).  The (TX + 2 RING) / 2 nodes of
// the colour in each of the TY + 2 RING rows are numbered row by row and thread t of the
// NT takes t, t + NT, ...: for windows of a few dozen nodes a row this keeps every lane
// busy, where a warp per row would leave up to half of them idle.  Nodes of one colour
// depend only on the other colour, so the order does not change the result.
template <typename R, int W, int TX, int TY, int NT, int RING, int COLOR>
__device__ __forceinline__ void half_sweep_flat(typename C2<R>::T* E0, typename C2<R>::T* E1,
                                                const typename C2<R>::T* R0,
                                                const typename C2<R>::T* R1, int gx0, int gy0,
                                                int x0, int y0, int n, R h2, R dinv)
{
    typedef typename C2<R>::T c2;
    typedef Planes<W> PL;
    constexpr int NX = (TX + 2 * RING) / 2, NY = TY + 2 * RING;
    static_assert(TX % 2 == 0, "whole colour pairs per row");
    c2* __restrict__ Ec = COLOR ? E1 : E0;
    const c2* __restrict__ Eo = COLOR ? E0 : E1;
    const c2* __restrict__ Rc = COLOR ? R1 : R0;
    const int xr = x0 - RING;
    for (int q = threadIdx.x; q < NX * NY; q += NT) {
        const int j = q / NX, i = q - j * NX;
        const int gy = y0 - RING + j;
        const int gx = xr + (((xr + gy) & 1) ^ COLOR) + 2 * i;
        if (gy < 1 || gy > n || gx < 1 || gx > n) continue;
        const int lx = gx - gx0, ly = gy - gy0;
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

// NS half-sweeps on rings RING, RING - 1, ..., RING - NS + 1, colours 0, 1, 0, ..., a
// barrier after each.
template <typename R, int W, int TX, int TY, int NT, int RING, int NS, int COLOR = 0>
__device__ __forceinline__ void sweeps_flat(typename C2<R>::T* E0, typename C2<R>::T* E1,
                                            const typename C2<R>::T* R0, const typename C2<R>::T* R1,
                                            int gx0, int gy0, int x0, int y0, int n, R h2, R dinv)
{
    if constexpr (NS > 0) {
        static_assert(RING >= 0, "rings down to the tile itself");
        half_sweep_flat<R, W, TX, TY, NT, RING, COLOR>(E0, E1, R0, R1, gx0, gy0, x0, y0, n, h2, dinv);
        __syncthreads();
        sweeps_flat<R, W, TX, TY, NT, RING - 1, NS - 1, COLOR ^ 1>(E0, E1, R0, R1, gx0, gy0, x0, y0, n, h2,
                                                                   dinv);
    }
}

}  // namespace
}  // namespace helm
