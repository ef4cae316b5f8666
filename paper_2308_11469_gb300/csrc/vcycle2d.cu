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
// The sweep counts are template parameters (1..4), so every extent is a compile-time
// constant; a warp walks a row (lanes along x), the 8 warps stride over rows.
//
// The node colours, the update formula and the transfer weights are those of the
// generic kernels (vcycle.cu), so both paths compute the same V-cycle; the shift sigma
// of the general cavity enters the local solve (diagonal 4 + sigma h^2) and the residual.
#include "launch.h"
#include "pdl.cuh"
#include "sweep2d.cuh"

namespace helm {
namespace {

constexpr int NT = SW_NT;
constexpr int NW = SW_NW;

template <typename R, int NU, int TX, int TY>
__global__ void __launch_bounds__(NT)
k_down2d(const InstDesc* __restrict__ insts, const InstState* __restrict__ st,
         const MgItem* __restrict__ items, int zero_mode)
{
    typedef typename C2<R>::T c2;
    constexpr int H = 2 * NU + 2;
    constexpr int W = TX + 2 * H, HH = TY + 2 * H;
    typedef Planes<W> PL;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // work item and level descriptors are written by the host before the launch: read them
    // before waiting for the predecessor kernel (overlaps its drain)
    const MgItem item = items[blockIdx.y];
    const LevelDesc L = insts[item.inst].lev[item.level];
    const LevelDesc C = insts[item.inst].lev[item.level + 1];
    const double sigma = insts[item.inst].sigma;
    pdl_wait();
    pdl_trigger();
    const InstState sv = st[item.inst];
    if (sv.status != HELM_ST_ACTIVE) return;
    const int n = L.n;
    const int ntx = (n + TX - 1) / TX;
    const int nty = (n + TY - 1) / TY;
    if ((int)blockIdx.x >= ntx * nty) return;
    const int x0 = 1 + (blockIdx.x % ntx) * TX;
    const int y0 = 1 + (blockIdx.x / ntx) * TY;
    c2* base = reinterpret_cast<c2*>(smem_raw);
    constexpr int PS = HH * PL::WH;                 // one colour plane
    c2* const E0 = base;
    c2* const E1 = base + PS;
    c2* const R0 = base + 2 * PS;
    c2* const R1 = base + 3 * PS;
    const int gx0 = x0 - H, gy0 = y0 - H;
    const int cpar = (gx0 + gy0) & 1;
    const bool zero = (zero_mode == 2) || (zero_mode == 1 && item.level > 0);
    const c2* __restrict__ ge = (const c2*)L.e;
    const c2* __restrict__ gr = (const c2*)lev_rhs(L, item.level, sv.it);
    const int P = L.pitch;
    const int lane = threadIdx.x & 31;
    // stage e (or zeros) and rhs with asynchronous copies: every load of the tile is in
    // flight at once; nodes outside the interior are zero-filled
    for (int q = threadIdx.x; q < W * HH; q += NT) {
        const int ly = q / W, lx = q - ly * W;
        const int gy = gy0 + ly;
        const bool yin = gy >= 1 && gy <= n;
        const int gx = gx0 + lx;
        const bool in = yin && gx >= 1 && gx <= n;
        const size_t g = in ? (size_t)gy * P + gx : 0;
        const int c = (lx + ly + cpar) & 1;
        const int o = PL::at(lx, ly);
        if (zero) (c ? E1 : E0)[o] = cz<c2>();
        else cp_async_elem<sizeof(c2)>((c ? E1 : E0) + o, ge + g, in);
        cp_async_elem<sizeof(c2)>((c ? R1 : R0) + o, gr + g, in);
    }
    cp_async_wait_all();
    __syncthreads();
    const R h2 = (R)(L.h * L.h);
    const R dinv = (R)L.dinv;                      // 1 / (4 + sigma h^2)
    const R sig = (R)sigma;
    sweeps_flat<R, W, TX, TY, NT, 2 * NU + 1, 2 * NU>(E0, E1, R0, R1, gx0, gy0, x0, y0, n, h2, dinv);
    // no pre-smoothing from a zero iterate: e2 stays zero (the ascent kernel knows it and
    // does not read it) and the residual is rhs itself
    const bool skip = (NU == 0) && zero;
    // smoothed iterate of the tile -> e2
    c2* __restrict__ ge2 = (c2*)L.e2;
    for (int ty = threadIdx.x >> 5; ty < TY && !skip; ty += NW) {
        const int gy = y0 + ty;
        if (gy > n) break;
#pragma unroll
        for (int tx = lane; tx < TX; tx += 32) {
            const int gx = x0 + tx;
            const int lx = tx + H, ly = ty + H;
            if (gx <= n) ge2[(size_t)gy * P + gx] = (((lx + ly + cpar) & 1) ? E1 : E0)[PL::at(lx, ly)];
        }
    }
    // residual on the tile plus a 1-node ring, in place of rhs (one colour at a time)
    const R ih2 = (R)1 / h2;
    if (!skip) {
        // both colours' nodes of the tile plus its ring, numbered colour by colour and row
        // by row over the threads ((TX + 2) / 2 of a colour in each of TY + 2 rows)
        constexpr int NX = (TX + 2) / 2, NY = TY + 2;
        for (int q = threadIdx.x; q < 2 * NX * NY; q += NT) {
            const int color = q >= NX * NY;
            const int qq = q - color * (NX * NY);
            const int jy = qq / NX, i = qq - jy * NX;
            const int gy = y0 - 1 + jy;
            const int gx = x0 - 1 + (((x0 - 1 + gy) & 1) ^ color) + 2 * i;
            if (gy < 1 || gy > n || gx < 1 || gx > n) continue;
            const c2* __restrict__ Ec = color ? E1 : E0;
            const c2* __restrict__ Eo = color ? E0 : E1;
            c2* __restrict__ Rc = color ? R1 : R0;
            const int ly = gy - gy0;
            const int lx = gx - gx0;
            const int o = PL::at(lx, ly);
            const c2 c = Ec[o];
            const c2 a = Eo[PL::at(lx - 1, ly)], b = Eo[PL::at(lx + 1, ly)];
            const c2 u = Eo[PL::at(lx, ly - 1)], d = Eo[PL::at(lx, ly + 1)];
            const c2 rr = Rc[o];
            c2 v;
            v.x = (rr.x - ((a.x + b.x + u.x + d.x) - (R)4 * c.x) * ih2) + sig * c.x;
            v.y = (rr.y - ((a.y + b.y + u.y + d.y) - (R)4 * c.y) * ih2) + sig * c.y;
            Rc[o] = v;
        }
    }
    __syncthreads();
    // full weighting at the coarse nodes owned by this tile (TX/2 x TY/2 of them)
    c2* __restrict__ cr = (c2*)C.rhs;
    const int nc = C.n;
    const int Xa = (x0 + 1) >> 1, Ya = (y0 + 1) >> 1;
    const int PC = C.pitch;
    for (int q = threadIdx.x; q < (TX / 2) * (TY / 2); q += NT) {
        const int cy = q / (TX / 2), cx = q - cy * (TX / 2);
        const int Y = Ya + cy;
        const int X = Xa + cx;
        if (Y > nc || X > nc) continue;
        const int lx = 2 * X - gx0, ly = 2 * Y - gy0;
        R ax = 0, ay = 0;
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy) {
            const R wy = (dy == 0) ? (R)2 : (R)1;
#pragma unroll
            for (int dx = -1; dx <= 1; ++dx) {
                const R wgt = wy * ((dx == 0) ? (R)2 : (R)1);
                const c2 r = (((lx + dx + ly + dy + cpar) & 1) ? R1 : R0)[PL::at(lx + dx, ly + dy)];
                ax += wgt * r.x;
                ay += wgt * r.y;
            }
        }
        c2 v;
        v.x = ax * (R)(1.0 / 16.0);
        v.y = ay * (R)(1.0 / 16.0);
        cr[(size_t)Y * PC + X] = v;
    }
}

template <typename R, int NU, int TX, int TY>
__global__ void __launch_bounds__(NT)
k_up2d(const InstDesc* __restrict__ insts, const InstState* __restrict__ st,
       const MgItem* __restrict__ items, int e2_mode)
{
    typedef typename C2<R>::T c2;
    constexpr int H = 2 * NU;
    constexpr int W = TX + 2 * H, HH = TY + 2 * H;
    constexpr int CW = W / 2 + 2, CH = HH / 2 + 2;
    typedef Planes<W> PL;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // work item and level descriptors are written by the host before the launch: read them
    // before waiting for the predecessor kernel (overlaps its drain)
    const MgItem item = items[blockIdx.y];
    const LevelDesc L = insts[item.inst].lev[item.level];
    const LevelDesc C = insts[item.inst].lev[item.level + 1];
    pdl_wait();
    pdl_trigger();
    const InstState sv = st[item.inst];
    if (sv.status != HELM_ST_ACTIVE) return;
    const int n = L.n;
    const int ntx = (n + TX - 1) / TX;
    const int nty = (n + TY - 1) / TY;
    if ((int)blockIdx.x >= ntx * nty) return;
    const int x0 = 1 + (blockIdx.x % ntx) * TX;
    const int y0 = 1 + (blockIdx.x / ntx) * TY;
    c2* base = reinterpret_cast<c2*>(smem_raw);
    constexpr int PS = HH * PL::WH;
    c2* const E0 = base;
    c2* const E1 = base + PS;
    c2* const R0 = base + 2 * PS;
    c2* const R1 = base + 3 * PS;
    c2* Cs = base + 4 * PS;
    const int gx0 = x0 - H, gy0 = y0 - H;
    const int cpar = (gx0 + gy0) & 1;
    // coarse window: X in [cx0, cx0 + CW), clipped to the padded coarse grid
    const int cx0 = max(gx0, 0) >> 1, cy0 = max(gy0, 0) >> 1;
    const int nc1 = C.n + 1;
    const c2* __restrict__ gce = (const c2*)C.e;
    const int PC = C.pitch;
    const int lane = threadIdx.x & 31;
    const c2* __restrict__ ge2 = (const c2*)L.e2;
    const c2* __restrict__ gr = (const c2*)lev_rhs(L, item.level, sv.it);
    const int P = L.pitch;
    // e2 is zero (not written by the descent) when the cycle has no pre-smoothing and the
    // level started from zero: e2_mode 2 = every level, 1 = the levels below the finest
    const bool e2z = (e2_mode == 2) || (e2_mode == 1 && item.level > 0);
    // stage the coarse window, e2 and rhs with asynchronous copies (zero-filled outside)
    // windows numbered row by row over the threads (rows of a few dozen nodes: a warp per
    // row would leave lanes idle)
    for (int q = threadIdx.x; q < CW * CH; q += NT) {
        const int cy = q / CW, cx = q - cy * CW;
        const int Y = cy0 + cy;
        const int X = cx0 + cx;
        const bool in = X <= nc1 && Y <= nc1;
        cp_async_elem<sizeof(c2)>(Cs + cy * CW + cx, gce + (in ? (size_t)Y * PC + X : 0), in);
    }
    for (int q = threadIdx.x; q < W * HH; q += NT) {
        const int ly = q / W, lx = q - ly * W;
        const int gy = gy0 + ly;
        const bool yin = gy >= 1 && gy <= n;
        const int gx = gx0 + lx;
        const bool in = yin && gx >= 1 && gx <= n;
        const size_t g = in ? (size_t)gy * P + gx : 0;
        const int c = (lx + ly + cpar) & 1;
        const int o = PL::at(lx, ly);
        if (e2z) (c ? E1 : E0)[o] = cz<c2>();
        else cp_async_elem<sizeof(c2)>((c ? E1 : E0) + o, ge2 + g, in);
        cp_async_elem<sizeof(c2)>((c ? R1 : R0) + o, gr + g, in);
    }
    cp_async_wait_all();
    __syncthreads();
    // correction: e2 + multilinear interpolation of the coarse iterate (interior nodes)
    for (int q = threadIdx.x; q < W * HH; q += NT) {
        const int ly = q / W, lx = q - ly * W;
        const int gy = gy0 + ly;
        if (gy < 1 || gy > n) continue;
        const int Y0 = (gy >> 1) - cy0, Y1 = ((gy + 1) >> 1) - cy0;
        const int gx = gx0 + lx;
        if (gx < 1 || gx > n) continue;
        const int X0 = (gx >> 1) - cx0, X1 = ((gx + 1) >> 1) - cx0;
        const c2 a = Cs[Y0 * CW + X0], b = Cs[Y0 * CW + X1];
        const c2 c = Cs[Y1 * CW + X0], d = Cs[Y1 * CW + X1];
        c2* Ep = (((lx + ly + cpar) & 1) ? E1 : E0) + PL::at(lx, ly);
        c2 v = *Ep;
        v.x += (R)0.25 * (((a.x + b.x) + c.x) + d.x);
        v.y += (R)0.25 * (((a.y + b.y) + c.y) + d.y);
        *Ep = v;
    }
    __syncthreads();
    const R h2 = (R)(L.h * L.h);
    const R dinv = (R)L.dinv;
    sweeps_flat<R, W, TX, TY, NT, 2 * NU - 1, 2 * NU>(E0, E1, R0, R1, gx0, gy0, x0, y0, n, h2, dinv);
    c2* __restrict__ ge = (c2*)L.e;
    for (int ty = threadIdx.x >> 5; ty < TY; ty += NW) {
        const int gy = y0 + ty;
        if (gy > n) break;
#pragma unroll
        for (int tx = lane; tx < TX; tx += 32) {
            const int gx = x0 + tx;
            const int lx = tx + H, ly = ty + H;
            if (gx <= n) ge[(size_t)gy * P + gx] = (((lx + ly + cpar) & 1) ? E1 : E0)[PL::at(lx, ly)];
        }
    }
}

// Descent step of a cycle without pre-smoothing from a zero iterate: the residual is rhs
// itself, so the coarse rhs is the full weighting of rhs -- no staging, no iterate.  One
// thread per coarse node (32 x 8 per CTA), its nine fine values read through L1; the
// weights and their order are those of k_down2d's restriction.
constexpr int RX = 32, RY = 8;

template <typename R>
__global__ void __launch_bounds__(RX * RY)
k_restrict_rhs2d(const InstDesc* __restrict__ insts, const InstState* __restrict__ st,
                 const MgItem* __restrict__ items)
{
    typedef typename C2<R>::T c2;
    const MgItem item = items[blockIdx.y];
    const LevelDesc L = insts[item.inst].lev[item.level];
    const LevelDesc C = insts[item.inst].lev[item.level + 1];
    pdl_wait();
    pdl_trigger();
    const InstState sv = st[item.inst];
    if (sv.status != HELM_ST_ACTIVE) return;
    const int nc = C.n;
    const int ntx = (nc + RX - 1) / RX;
    if ((int)blockIdx.x >= ntx * ((nc + RY - 1) / RY)) return;
    const int X = 1 + (blockIdx.x % ntx) * RX + (threadIdx.x % RX);
    const int Y = 1 + (blockIdx.x / ntx) * RY + (threadIdx.x / RX);
    if (X > nc || Y > nc) return;
    const c2* __restrict__ gr = (const c2*)lev_rhs(L, item.level, sv.it);
    const size_t P = L.pitch;
    const size_t o = (size_t)(2 * Y) * P + 2 * X;
    R ax = 0, ay = 0;
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy) {
        const R wy = (dy == 0) ? (R)2 : (R)1;
#pragma unroll
        for (int dx = -1; dx <= 1; ++dx) {
            const R wgt = wy * ((dx == 0) ? (R)2 : (R)1);
            const c2 r = __ldg(gr + (o + (ptrdiff_t)dy * (ptrdiff_t)P + dx));
            ax += wgt * r.x;
            ay += wgt * r.y;
        }
    }
    c2 v;
    v.x = ax * (R)(1.0 / 16.0);
    v.y = ay * (R)(1.0 / 16.0);
    ((c2*)C.rhs)[(size_t)Y * C.pitch + X] = v;
}

// Two such descent steps in one launch: level l+1's rhs = full weighting of level l's rhs,
// level l+2's rhs = full weighting of that (same weights, order and scaling as
// k_restrict_rhs2d, so the values are the same).  A CTA owns a 16 x 16 tile of level l+2:
// it stages the 68 x 68 window of level l's rhs the tile depends on (16-byte copies from a
// 16-byte aligned column), forms the 33 x 33 level-(l+1) nodes the tile reads, writes the
// 32 x 32 of them it owns (level l+1 columns 32 i + 1 .. 32 i + 32 for tile column i) and
// the tile.
constexpr int R2T = 16;                    // level l+2 tile edge
constexpr int R2W1 = 2 * R2T + 1;          // level l+1 window edge
constexpr int R2W0 = 4 * R2T + 4;          // level l window edge
constexpr int R2NT = 256;
static_assert(R2T * R2T <= R2NT, "a thread per node of the level l+2 tile");

template <typename R> constexpr size_t restrict2_bytes()
{
    return ((size_t)R2W0 * R2W0 + (size_t)R2W1 * R2W1) * 2 * sizeof(R);
}

template <typename R>
__global__ void __launch_bounds__(R2NT)
k_restrict2_rhs2d(const InstDesc* __restrict__ insts, const InstState* __restrict__ st,
                  const MgItem* __restrict__ items)
{
    typedef typename C2<R>::T c2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    c2* W0 = reinterpret_cast<c2*>(smem_raw);           // level l window
    c2* W1 = W0 + R2W0 * R2W0;                           // level l+1 window
    const MgItem item = items[blockIdx.y];
    const LevelDesc L0 = insts[item.inst].lev[item.level];
    const LevelDesc L1 = insts[item.inst].lev[item.level + 1];
    const LevelDesc L2 = insts[item.inst].lev[item.level + 2];
    pdl_wait();
    pdl_trigger();
    const InstState sv = st[item.inst];
    if (sv.status != HELM_ST_ACTIVE) return;
    const int n0 = L0.n, n1 = L1.n, n2 = L2.n;
    const int ntx = (n2 + R2T - 1) / R2T;
    if ((int)blockIdx.x >= ntx * ntx) return;
    const int X2a = 1 + (blockIdx.x % ntx) * R2T, Y2a = 1 + (blockIdx.x / ntx) * R2T;
    const int c0 = 4 * X2a - 4, r0 = 4 * Y2a - 4;       // level l window origin
    const c2* __restrict__ g0 = (const c2*)lev_rhs(L0, item.level, sv.it);
    const int P0 = L0.pitch;
    // stage: 16-byte chunks (two complex64 or one complex128), zero outside the array
    constexpr int EPC = 16 / (int)sizeof(c2);             // elements per chunk
    constexpr int CPR = R2W0 / EPC;                       // chunks per window row
    for (int q = threadIdx.x; q < R2W0 * CPR; q += R2NT) {
        const int r = q / CPR, cc = (q % CPR) * EPC;
        const int gy = r0 + r, gx = c0 + cc;
        const bool in = gy <= n0 + 1 && gx < P0;
        const c2* src = g0 + (in ? (size_t)gy * P0 + gx : 0);
        const unsigned d = (unsigned)__cvta_generic_to_shared(W0 + r * R2W0 + cc);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(in ? 16 : 0)
                     : "memory");
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    __syncthreads();
    // level l+1 window: node (2 X2a - 1 + x1, 2 Y2a - 1 + y1); its fine node (2 X1 + dx, ...)
    // is window element (2 x1 + 2 + dx, 2 y1 + 2 + dy)
    c2* __restrict__ g1 = (c2*)L1.rhs;
    const int P1 = L1.pitch;
    for (int q = threadIdx.x; q < R2W1 * R2W1; q += R2NT) {
        const int y1 = q / R2W1, x1 = q % R2W1;
        const int X1 = 2 * X2a - 1 + x1, Y1 = 2 * Y2a - 1 + y1;
        c2 v;
        v.x = 0;
        v.y = 0;
        if (X1 <= n1 && Y1 <= n1) {
            R ax = 0, ay = 0;
#pragma unroll
            for (int dy = -1; dy <= 1; ++dy) {
                const R wy = (dy == 0) ? (R)2 : (R)1;
#pragma unroll
                for (int dx = -1; dx <= 1; ++dx) {
                    const R wgt = wy * ((dx == 0) ? (R)2 : (R)1);
                    const c2 r = W0[(2 * y1 + 2 + dy) * R2W0 + 2 * x1 + 2 + dx];
                    ax += wgt * r.x;
                    ay += wgt * r.y;
                }
            }
            v.x = ax * (R)(1.0 / 16.0);
            v.y = ay * (R)(1.0 / 16.0);
            if (x1 < 2 * R2T && y1 < 2 * R2T) g1[(size_t)Y1 * P1 + X1] = v;
        }
        W1[q] = v;
    }
    __syncthreads();
    // the level l+2 tile: node (X2a + x2, Y2a + y2) reads window element (2 x2 + 1 + dx, ...)
    c2* __restrict__ g2 = (c2*)L2.rhs;
    const int P2 = L2.pitch;
    const int x2 = threadIdx.x % R2T, y2 = threadIdx.x / R2T;
    const int X2 = X2a + x2, Y2 = Y2a + y2;
    if (y2 < R2T && X2 <= n2 && Y2 <= n2) {
        R ax = 0, ay = 0;
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy) {
            const R wy = (dy == 0) ? (R)2 : (R)1;
#pragma unroll
            for (int dx = -1; dx <= 1; ++dx) {
                const R wgt = wy * ((dx == 0) ? (R)2 : (R)1);
                const c2 r = W1[(2 * y2 + 1 + dy) * R2W1 + 2 * x2 + 1 + dx];
                ax += wgt * r.x;
                ay += wgt * r.y;
            }
        }
        c2 v;
        v.x = ax * (R)(1.0 / 16.0);
        v.y = ay * (R)(1.0 / 16.0);
        g2[(size_t)Y2 * P2 + X2] = v;
    }
}

template <int NU, int TX, int TY> constexpr size_t down_bytes(size_t eb) {
    return 2 * (size_t)(TX + 2 * (2 * NU + 2)) * (TY + 2 * (2 * NU + 2)) * eb;
}
template <int NU, int TX, int TY> constexpr size_t up_bytes(size_t eb) {
    return ((size_t)2 * (TX + 4 * NU) * (TY + 4 * NU) +
            (size_t)((TX + 4 * NU) / 2 + 2) * ((TY + 4 * NU) / 2 + 2)) * eb;
}

// tile shapes: 0 = 64 x 32, 1 = 32 x 16 (levels <= 511 whose launch would otherwise leave
// the GPU under-filled: a lone instance's coarser levels still spread over many SMs)
template <int S> struct Shape;
template <> struct Shape<0> { static constexpr int X = 64, Y = 32; };
template <> struct Shape<1> { static constexpr int X = 32, Y = 16; };

template <typename R, int NU, int S>
cudaError_t set_attrs_s()
{
    constexpr int X = Shape<S>::X, Y = Shape<S>::Y;
    cudaError_t e = cudaFuncSetAttribute(k_down2d<R, NU, X, Y>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)down_bytes<NU, X, Y>(sizeof(R) * 2));
    if (e != cudaSuccess) return e;
    if ((e = max_carveout(k_down2d<R, NU, X, Y>)) != cudaSuccess) return e;
    if ((e = max_carveout(k_up2d<R, NU, X, Y>)) != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_up2d<R, NU, X, Y>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)up_bytes<NU, X, Y>(sizeof(R) * 2));
}

template <typename R, int NU>
cudaError_t set_attrs()
{
    cudaError_t e = set_attrs_s<R, NU, 0>();
    if (e != cudaSuccess) return e;
    return set_attrs_s<R, NU, 1>();
}

template <typename R>
cudaError_t set_all()
{
    cudaError_t e;
    if ((e = max_carveout(k_restrict_rhs2d<R>)) != cudaSuccess) return e;
    if ((e = max_carveout(k_restrict2_rhs2d<R>)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_restrict2_rhs2d<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)restrict2_bytes<R>())) != cudaSuccess)
        return e;
    if ((e = set_attrs<R, 0>()) != cudaSuccess) return e;
    if ((e = set_attrs<R, 1>()) != cudaSuccess) return e;
    if ((e = set_attrs<R, 2>()) != cudaSuccess) return e;
    if ((e = set_attrs<R, 3>()) != cudaSuccess) return e;
    return set_attrs<R, 4>();
}

template <typename R, int NU, int S>
void down_s(dim3 g, const InstDesc* insts, const InstState* st, const MgItem* items, int zero_mode,
            cudaStream_t s)
{
    constexpr int X = Shape<S>::X, Y = Shape<S>::Y;
    launch_k(k_down2d<R, NU, X, Y>, g, dim3(NT), down_bytes<NU, X, Y>(sizeof(R) * 2), s, insts, st,
             items, zero_mode);
}

template <typename R, int NU, int S>
void up_s(dim3 g, const InstDesc* insts, const InstState* st, const MgItem* items, int e2_mode,
          cudaStream_t s)
{
    constexpr int X = Shape<S>::X, Y = Shape<S>::Y;
    launch_k(k_up2d<R, NU, X, Y>, g, dim3(NT), up_bytes<NU, X, Y>(sizeof(R) * 2), s, insts, st, items,
             e2_mode);
}

template <typename R, int S>
cudaError_t down(int nu, dim3 g, const InstDesc* insts, const InstState* st, const MgItem* items,
                 int zero_mode, cudaStream_t s)
{
    switch (nu) {
    case 0: down_s<R, 0, S>(g, insts, st, items, zero_mode, s); break;
    case 1: down_s<R, 1, S>(g, insts, st, items, zero_mode, s); break;
    case 2: down_s<R, 2, S>(g, insts, st, items, zero_mode, s); break;
    case 3: down_s<R, 3, S>(g, insts, st, items, zero_mode, s); break;
    case 4: down_s<R, 4, S>(g, insts, st, items, zero_mode, s); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <typename R, int S>
cudaError_t up(int nu, dim3 g, const InstDesc* insts, const InstState* st, const MgItem* items,
               int e2_mode, cudaStream_t s)
{
    switch (nu) {
    case 0: up_s<R, 0, S>(g, insts, st, items, e2_mode, s); break;
    case 1: up_s<R, 1, S>(g, insts, st, items, e2_mode, s); break;
    case 2: up_s<R, 2, S>(g, insts, st, items, e2_mode, s); break;
    case 3: up_s<R, 3, S>(g, insts, st, items, e2_mode, s); break;
    case 4: up_s<R, 4, S>(g, insts, st, items, e2_mode, s); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace

int tile_shape2d(int n) { return n <= 511 ? 1 : 0; }

int tiles2d_for(int n, int shape)
{
    const int X = shape ? Shape<1>::X : Shape<0>::X;
    const int Y = shape ? Shape<1>::Y : Shape<0>::Y;
    return ((n + X - 1) / X) * ((n + Y - 1) / Y);
}

int tiles2d(int n) { return tiles2d_for(n, tile_shape2d(n)); }

cudaError_t setup_2d(int prec) { return prec == 0 ? set_all<double>() : set_all<float>(); }

// shape: the tile shape of every item of the launch (tile_shape2d of the largest level)
cudaError_t launch_down2d(int prec, const InstDesc* insts, const InstState* st, const MgItem* items,
                          int nitems, int max_tiles, int nu1, int zero_mode, int shape, cudaStream_t s,
                          int nmax)
{
    if (nu1 == 0 && zero_mode == 2 && nmax > 0) {
        // every iterate of the launch is zero: restriction of rhs alone
        const int nc = (nmax - 1) / 2;
        dim3 gr(((nc + RX - 1) / RX) * ((nc + RY - 1) / RY), nitems);
        if (prec == 0) launch_k(k_restrict_rhs2d<double>, gr, dim3(RX * RY), 0, s, insts, st, items);
        else launch_k(k_restrict_rhs2d<float>, gr, dim3(RX * RY), 0, s, insts, st, items);
        return cudaGetLastError();
    }
    dim3 g(max_tiles, nitems);
    if (shape) return prec == 0 ? down<double, 1>(nu1, g, insts, st, items, zero_mode, s)
                                : down<float, 1>(nu1, g, insts, st, items, zero_mode, s);
    return prec == 0 ? down<double, 0>(nu1, g, insts, st, items, zero_mode, s)
                     : down<float, 0>(nu1, g, insts, st, items, zero_mode, s);
}

cudaError_t launch_restrict2_2d(int prec, const InstDesc* insts, const InstState* st, const MgItem* items,
                                int nitems, int nmax, cudaStream_t s)
{
    const int n2 = ((nmax - 1) / 2 - 1) / 2;
    if (n2 < 1) return cudaErrorInvalidValue;
    const int t = (n2 + R2T - 1) / R2T;
    dim3 g(t * t, nitems);
    if (prec == 0) launch_k(k_restrict2_rhs2d<double>, g, dim3(R2NT), restrict2_bytes<double>(), s, insts, st, items);
    else launch_k(k_restrict2_rhs2d<float>, g, dim3(R2NT), restrict2_bytes<float>(), s, insts, st, items);
    return cudaGetLastError();
}

cudaError_t launch_up2d(int prec, const InstDesc* insts, const InstState* st, const MgItem* items,
                        int nitems, int max_tiles, int nu2, int shape, int e2_mode, cudaStream_t s)
{
    dim3 g(max_tiles, nitems);
    if (shape) return prec == 0 ? up<double, 1>(nu2, g, insts, st, items, e2_mode, s)
                                : up<float, 1>(nu2, g, insts, st, items, e2_mode, s);
    return prec == 0 ? up<double, 0>(nu2, g, insts, st, items, e2_mode, s)
                     : up<float, 0>(nu2, g, insts, st, items, e2_mode, s);
}

}  // namespace helm
