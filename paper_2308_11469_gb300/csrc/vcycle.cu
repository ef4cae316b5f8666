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
// 3D half-sweep marching in z with the planes staged by asynchronous copies
// ---------------------------------------------------------------------------
// The same half-sweep as k_rbgs<3, R> mode 0 (same operands, same summation order), for
// levels whose colour-split rows fit shared memory.  A CTA owns TY rows (y) over a chunk of
// planes (z).  For every row (y', z') around them it needs one half of the row: the half
// holding the other colour (x parity 1 - p(y', z'), p = the parity of the updated x in that
// row); for its own rows the rhs half of the updated colour.  Plane by plane these halves are
// copied (16-byte cp.async, whole halves: pitch / 2 elements, 16-byte aligned) into rings:
// other-colour halves of rows y0-1 .. y0+TY of planes p-1 .. p+L+1 (L planes in flight) and
// rhs halves of rows y0 .. y0+TY-1 of planes p .. p+L.  In those halves the node at x of the
// updated colour finds its y- and z-neighbours at the same index j (x = 2j + p... / 2j) and its
// x-neighbours at j, j+1 (odd x) or j-1, j (even x).  No shared-memory word is written by the
// sweep; results go straight to global memory.
template <typename R> struct Rb3p {
    static constexpr int TY = sizeof(R) == 4 ? 8 : 4;      // rows per CTA (a warp per row)
    static constexpr int L = 1;                            // planes in flight
    static constexpr int OS = L + 3, RS = L + 1;           // ring slots
    static constexpr int MAX_HP = 264;                     // pitch / 2 of n = 511
    static size_t bytes(int hp) {
        return (size_t)(OS * (TY + 2) + RS * TY) * hp * sizeof(typename C2<R>::T);
    }
};

template <typename R>
__global__ void __launch_bounds__(32 * Rb3p<R>::TY)
k_rbgs3p(const InstDesc* __restrict__ insts, const InstState* __restrict__ st,
         const MgItem* __restrict__ items, int color, int zchunk)
{
    typedef typename C2<R>::T c2;
    typedef Rb3p<R> K;
    constexpr int TY = K::TY, L = K::L;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const MgItem item = items[blockIdx.y];
    const LevelDesc Lv = insts[item.inst].lev[item.level];
    pdl_wait();
    pdl_trigger();
    const InstState sv = st[item.inst];
    if (sv.status != HELM_ST_ACTIVE) return;
    const int n = Lv.n;
    const int nyb = (n + TY - 1) / TY, nzc = (n + zchunk - 1) / zchunk;
    if ((int)blockIdx.x >= nyb * nzc) return;
    const int y0 = 1 + (int)(blockIdx.x % nyb) * TY;
    const int z0 = 1 + (int)(blockIdx.x / nyb) * zchunk;
    const int z1 = min(z0 + zchunk, n + 1);                // own planes [z0, z1)
    const int HP = Lv.pitch >> 1;
    const size_t PR = (size_t)Lv.pitch, PL = (size_t)Lv.pitch * Lv.rows;
    c2* __restrict__ e = (c2*)Lv.e;
    const c2* __restrict__ r = (const c2*)lev_rhs(Lv, item.level, sv.it);
    c2* O = reinterpret_cast<c2*>(smem_raw);               // [OS][TY + 2][HP]
    c2* Rs = O + K::OS * (TY + 2) * HP;                    // [RS][TY][HP]
    constexpr int EPC = 16 / (int)sizeof(c2);               // elements per 16-byte chunk
    const int CPR = HP / EPC;                               // chunks per half row
    // copies: a warp per half row, its lanes over the row's 16-byte chunks (no division)
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // other-colour halves of rows y0-1 .. y0+TY of plane zp (zero past the last wall row)
    auto stage_o = [&](int zp) {
        c2* dst = O + (zp % K::OS) * (TY + 2) * HP;
        for (int i = w; i < TY + 2; i += TY) {
            const int yy = y0 - 1 + i;
            const bool in = yy <= n + 1;
            const int half = ((color + yy + zp) & 1) ? 0 : HP;   // the other colour's x parity
            const c2* src = in ? e + zp * PL + yy * PR + half : e;
            const unsigned d = (unsigned)__cvta_generic_to_shared(dst + i * HP);
            for (int c = lane; c < CPR; c += 32)
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d + 16 * c),
                             "l"(src + (in ? EPC * c : 0)), "r"(in ? 16 : 0) : "memory");
        }
    };
    // rhs halves (updated colour) of rows y0 .. y0+TY-1 of plane zp
    auto stage_r = [&](int zp) {
        c2* dst = Rs + (zp % K::RS) * TY * HP;
        const int yy = y0 + w;
        const bool in = yy <= n;
        const int half = ((color + yy + zp) & 1) ? HP : 0;
        const c2* src = in ? r + zp * PL + yy * PR + half : r;
        const unsigned d = (unsigned)__cvta_generic_to_shared(dst + w * HP);
        for (int c = lane; c < CPR; c += 32)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d + 16 * c),
                         "l"(src + (in ? EPC * c : 0)), "r"(in ? 16 : 0) : "memory");
    };
    auto commit = []() { asm volatile("cp.async.commit_group;\n" ::: "memory"); };
    // group of plane p: the other-colour halves of plane p + 1 and the rhs of plane p; before
    // them the halves of planes z0 - 1 and z0
    stage_o(z0 - 1);
    stage_o(z0);
    commit();
    for (int p = z0; p < z0 + L; ++p) {
        if (p < z1) {
            stage_o(p + 1);
            stage_r(p);
        }
        commit();
    }
    const R h2 = (R)(Lv.h * Lv.h);
    const R inv = (R)Lv.dinv;
    const int y = y0 + w;
    const int jmax = (n - 1) >> 1;
    for (int p = z0; p < z1; ++p) {
        if (p + L < z1) {
            stage_o(p + L + 1);
            stage_r(p + L);
        }
        commit();
        asm volatile("cp.async.wait_group %0;\n" ::"n"(L) : "memory");
        __syncthreads();
        if (y <= n) {
            const int px = (color + y + p) & 1;           // parity of the updated x
            const c2* oc = O + (p % K::OS) * (TY + 2) * HP + (w + 1) * HP;
            const c2* on = O + ((p - 1) % K::OS) * (TY + 2) * HP + (w + 1) * HP;
            const c2* op = O + ((p + 1) % K::OS) * (TY + 2) * HP + (w + 1) * HP;
            const c2* rr_ = Rs + (p % K::RS) * TY * HP + w * HP;
            c2* out = e + p * PL + y * PR + (px ? HP : 0);
#pragma unroll 4
            for (int j = lane + (px ? 0 : 1); j <= jmax; j += 32) {
                const int xa = px ? j : j - 1;                 // x - 1 in the other half
                const c2 a = oc[xa], b = oc[xa + 1];
                const c2 c = oc[j - HP], d = oc[j + HP];      // rows y - 1, y + 1
                R sx = a.x + b.x + c.x + d.x;
                R sy = a.y + b.y + c.y + d.y;
                const c2 f = on[j], g = op[j];
                sx += f.x + g.x;
                sy += f.y + g.y;
                const c2 rv = rr_[j];
                c2 v;
                v.x = (sx - h2 * rv.x) * inv;
                v.y = (sy - h2 * rv.y) * inv;
                out[j] = v;
            }
        }
        __syncthreads();
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

// 3D restriction of the rhs alone (a zero iterate, modes 2 / 1) marching in z: a CTA owns
// TYC coarse rows over a chunk of coarse planes; the fine rows 2 Y0 - 1 .. 2 Y0 + 2 TYC - 1 of
// the fine planes 2 Z - 1 .. 2 Z + 1 are staged whole (16-byte cp.async) in a ring of five
// fine planes (three in use, the next coarse plane's two in flight); the weights and the
// order of the 27-term sums are k_restrict's.
template <typename R> struct Rs3p {
    static constexpr int TYC = 4;                          // coarse rows per CTA
    static constexpr int NT = 256;                         // two warps per coarse row
    static constexpr int NS = 5;                           // fine-plane slots
    static constexpr int MAX_P = 528;                      // pitch of n = 511
    static size_t bytes(int pitch) {
        return (size_t)NS * (2 * TYC + 1) * pitch * sizeof(typename C2<R>::T);
    }
};

template <typename R>
__global__ void __launch_bounds__(Rs3p<R>::NT)
k_restrict3p(const InstDesc* __restrict__ insts, const InstState* __restrict__ st,
             const MgItem* __restrict__ items, int zchunk)
{
    typedef typename C2<R>::T c2;
    typedef Rs3p<R> K;
    constexpr int TYC = K::TYC, FR = 2 * TYC + 1;         // fine rows per plane slot
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const MgItem item = items[blockIdx.y];
    const LevelDesc F = insts[item.inst].lev[item.level];
    const LevelDesc C = insts[item.inst].lev[item.level + 1];
    pdl_wait();
    pdl_trigger();
    const InstState sv = st[item.inst];
    if (sv.status != HELM_ST_ACTIVE) return;
    const int n = F.n, nc = C.n;
    const int nyb = (nc + TYC - 1) / TYC, nzc = (nc + zchunk - 1) / zchunk;
    if ((int)blockIdx.x >= nyb * nzc) return;
    const int Y0 = 1 + (int)(blockIdx.x % nyb) * TYC;
    const int Z0 = 1 + (int)(blockIdx.x / nyb) * zchunk;
    const int Z1 = min(Z0 + zchunk, nc + 1);               // own coarse planes [Z0, Z1)
    const int P = F.pitch, HP = P >> 1;
    const size_t PR = (size_t)P, PL = (size_t)P * F.rows;
    const c2* __restrict__ r = (const c2*)lev_rhs(F, item.level, sv.it);
    c2* W = reinterpret_cast<c2*>(smem_raw);               // [NS][FR][P]
    constexpr int EPC = 16 / (int)sizeof(c2);
    const int CPR = P / EPC;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int y0f = 2 * Y0 - 1;                            // first fine row of a slot
    // fine plane f: rows y0f .. y0f + FR - 1 whole (zero past the last wall row), a warp per row
    auto stage = [&](int f) {
        c2* dst = W + (f % K::NS) * FR * P;
        for (int i = w; i < FR; i += K::NT / 32) {
            const int yy = y0f + i;
            const bool in = yy <= n + 1;
            const c2* src = in ? r + f * PL + yy * PR : r;
            const unsigned d = (unsigned)__cvta_generic_to_shared(dst + i * P);
            for (int c = lane; c < CPR; c += 32)
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d + 16 * c),
                             "l"(src + (in ? EPC * c : 0)), "r"(in ? 16 : 0) : "memory");
        }
    };
    auto commit = []() { asm volatile("cp.async.commit_group;\n" ::: "memory"); };
    stage(2 * Z0 - 1);
    stage(2 * Z0);
    stage(2 * Z0 + 1);
    commit();
    if (Z0 + 1 < Z1) {
        stage(2 * Z0 + 2);
        stage(2 * Z0 + 3);
    }
    commit();
    c2* __restrict__ cr = (c2*)C.rhs;
    const size_t PRc = (size_t)C.pitch, PLc = (size_t)C.pitch * C.rows;
    const R scale = (R)(1.0 / 64.0);
    const int cy = w >> 1;                                  // coarse row of the warp
    const int Y = Y0 + cy;
    for (int Z = Z0; Z < Z1; ++Z) {
        asm volatile("cp.async.wait_group 1;\n" ::: "memory");
        __syncthreads();
        if (Y <= nc) {
            for (int X = 1 + lane + 32 * (w & 1); X <= nc; X += 64) {
                R ax = 0, ay = 0;
#pragma unroll
                for (int dz = -1; dz <= 1; ++dz) {
                    const R wz = (dz == 0) ? (R)2 : (R)1;
                    const c2* pl = W + ((2 * Z + dz) % K::NS) * FR * P;
#pragma unroll
                    for (int dy = -1; dy <= 1; ++dy) {
                        const R wy = (dy == 0) ? (R)2 : (R)1;
                        const c2* row = pl + (2 * cy + 1 + dy) * P;   // fine row 2Y + dy
#pragma unroll
                        for (int dx = -1; dx <= 1; ++dx) {
                            const R wgt = wz * wy * ((dx == 0) ? (R)2 : (R)1);
                            const int x = 2 * X + dx;
                            const c2 rr = row[(x & 1) ? HP + (x >> 1) : (x >> 1)];
                            ax += wgt * rr.x;
                            ay += wgt * rr.y;
                        }
                    }
                }
                c2 v;
                v.x = ax * scale;
                v.y = ay * scale;
                cr[Z * PLc + Y * PRc + xslot<3>(X, C.pitch)] = v;
            }
        }
        __syncthreads();
        if (Z + 2 < Z1) {
            stage(2 * Z + 4);
            stage(2 * Z + 5);
        }
        commit();
    }
}

// ---------------------------------------------------------------------------
// Multilinear prolongation + correction
// ---------------------------------------------------------------------------
// mode 2 / 1: the fine iterate is zero on every level / on levels > 0 (no pre-smoothing
// from a zero iterate): e := interpolation instead of e += interpolation.  skip0: the next
// operation is a half-sweep of colour 0, which overwrites every colour-0 node without
// reading its value: only colour-1 nodes are corrected.
template <int D, typename R>
__global__ void __launch_bounds__(256)
k_prolong(const InstDesc* __restrict__ insts, const InstState* __restrict__ st,
          const MgItem* __restrict__ items, int mode, int skip0)
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
            if (skip0 && ((x + y + z) & 1) == 0) continue;
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
    if (D == 3 && sizeof(R) == 4) {                        // the z-marching forms are complex64 only
        if ((e = max_carveout(k_restrict3p<R>)) != cudaSuccess) return e;
        if ((e = cudaFuncSetAttribute(k_restrict3p<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)Rs3p<R>::bytes(Rs3p<float>::MAX_P))) != cudaSuccess)
            return e;
        if ((e = max_carveout(k_rbgs3p<R>)) != cudaSuccess) return e;
        if ((e = cudaFuncSetAttribute(k_rbgs3p<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)Rb3p<R>::bytes(Rb3p<float>::MAX_HP))) != cudaSuccess)
            return e;
    }
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
                        cudaStream_t s, int nmax)
{
    // 3D plain half-sweeps of levels 127 .. 511: the plane-marching form
    const int hp = (nmax + 2 + 15) / 16 * 8;
    if (D == 3 && prec != 0 && mode == 0 && nmax >= 127 && hp <= Rb3p<float>::MAX_HP) {
        const int ty = prec == 0 ? Rb3p<double>::TY : Rb3p<float>::TY;
        const size_t sm = prec == 0 ? Rb3p<double>::bytes(hp) : Rb3p<float>::bytes(hp);
        const int per_sm = (int)(227 * 1024 / (sm + 1024));
        const int nyb = (nmax + ty - 1) / ty;
        // z chunks so that the launch is about one wave of resident CTAs
        int nzc = (152 * (per_sm < 1 ? 1 : per_sm)) / (nyb * nitems);
        nzc = nzc < 1 ? 1 : (nzc > nmax / 4 ? nmax / 4 : nzc);     // at least 4 planes a CTA
        const int zchunk = (nmax + nzc - 1) / nzc;
        nzc = (nmax + zchunk - 1) / zchunk;
        dim3 g(nyb * nzc, nitems);
        if (prec == 0) launch_k(k_rbgs3p<double>, g, dim3(32 * ty), sm, s, insts, st, items, color, zchunk);
        else launch_k(k_rbgs3p<float>, g, dim3(32 * ty), sm, s, insts, st, items, color, zchunk);
        return cudaGetLastError();
    }
    dim3 g = mg_grid(work, nitems);
    if (D == 2 && prec == 0) launch_k(k_rbgs<2, double>, dim3(g), dim3(256), 0, s, insts, st, items, color, mode);
    else if (D == 2) launch_k(k_rbgs<2, float>, dim3(g), dim3(256), 0, s, insts, st, items, color, mode);
    else if (prec == 0) launch_k(k_rbgs<3, double>, dim3(g), dim3(256), 0, s, insts, st, items, color, mode);
    else launch_k(k_rbgs<3, float>, dim3(g), dim3(256), 0, s, insts, st, items, color, mode);
    return cudaGetLastError();
}

cudaError_t launch_restrict(int D, int prec, const InstDesc* insts, const InstState* st,
                            const MgItem* items, int nitems, int work, cudaStream_t s, int mode, int nmax)
{
    // 3D complex64 restriction of the rhs alone (every iterate of the launch zero) from fine
    // levels 127 .. 511: the z-marching form
    const int pitch = (nmax + 2 + 15) / 16 * 16;
    if (D == 3 && prec != 0 && mode == 2 && nmax >= 127 && pitch <= Rs3p<float>::MAX_P) {
        const int nc = (nmax - 1) / 2;
        const size_t sm = Rs3p<float>::bytes(pitch);
        const int per_sm = (int)(227 * 1024 / (sm + 1024));
        const int nyb = (nc + Rs3p<float>::TYC - 1) / Rs3p<float>::TYC;
        int nzc = (152 * (per_sm < 1 ? 1 : per_sm)) / (nyb * nitems);
        nzc = nzc < 1 ? 1 : (nzc > nc / 4 ? nc / 4 : nzc);      // at least 4 coarse planes a CTA
        const int zchunk = (nc + nzc - 1) / nzc;
        nzc = (nc + zchunk - 1) / zchunk;
        launch_k(k_restrict3p<float>, dim3(nyb * nzc, nitems), dim3(Rs3p<float>::NT), sm, s, insts, st, items,
                 zchunk);
        return cudaGetLastError();
    }
    dim3 g = mg_grid(work, nitems);
    if (D == 2 && prec == 0) launch_k(k_restrict<2, double>, dim3(g), dim3(256), 0, s, insts, st, items, mode);
    else if (D == 2) launch_k(k_restrict<2, float>, dim3(g), dim3(256), 0, s, insts, st, items, mode);
    else if (prec == 0) launch_k(k_restrict<3, double>, dim3(g), dim3(256), 0, s, insts, st, items, mode);
    else launch_k(k_restrict<3, float>, dim3(g), dim3(256), 0, s, insts, st, items, mode);
    return cudaGetLastError();
}

cudaError_t launch_prolong(int D, int prec, const InstDesc* insts, const InstState* st,
                           const MgItem* items, int nitems, int work, cudaStream_t s, int mode, int skip0)
{
    dim3 g = mg_grid(work, nitems);
    if (D == 2 && prec == 0) launch_k(k_prolong<2, double>, dim3(g), dim3(256), 0, s, insts, st, items, mode, skip0);
    else if (D == 2) launch_k(k_prolong<2, float>, dim3(g), dim3(256), 0, s, insts, st, items, mode, skip0);
    else if (prec == 0) launch_k(k_prolong<3, double>, dim3(g), dim3(256), 0, s, insts, st, items, mode, skip0);
    else launch_k(k_prolong<3, float>, dim3(g), dim3(256), 0, s, insts, st, items, mode, skip0);
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
