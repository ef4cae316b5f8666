// Shared device-side definitions of the Helmholtz Poisson-iteration library.
//
// Layouts
//  * outer arrays (caller memory, FP64): u padded (n+2)^D complex128, tight rows;
//    f interior n^D complex128; g padded (n+2)^D complex128 (ring = Dirichlet data).
//  * multigrid level arrays (library memory): padded (n_l+2)^D with the x pitch rounded
//    up to a multiple of 16 elements, so every row starts 128/256-byte aligned; the ring
//    of e is kept zero (homogeneous Dirichlet for the Poisson increments, Eq. (2.7) for
//    n >= 1), rhs rows use the same indexing (its ring is never read).  In 3D each x-row
//    is stored colour-split: its even-x nodes first (slot x/2), then its odd-x nodes (slot
//    pitch/2 + x/2); one colour of a row, and the other colour of the rows around it, are
//    then contiguous, so a red-black half-sweep reads and writes whole sectors (xslot).
//  * complex numbers are interleaved {re, im} pairs (float2 / double2).  The inner
//    operator is real, so the real and imaginary parts are two independent lanes of the
//    same real stencil (Eq. (2.5) with p = 0: the two chains do not couple).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define HELM_MAXLEV 16

// Instance status values kept on the device.  Non-negative values < 100 and negative
// values are the public helm_status outcomes; ACTIVE means "still iterating".
#define HELM_ST_ACTIVE 100
#define HELM_ST_IDLE 101

namespace helm {

struct LevelDesc {
    int n;        // interior nodes per axis, 2^(m-l) - 1
    int pitch;    // elements per x row (>= n + 2, multiple of 16)
    int rows;     // n + 2 rows per z plane
    int pad_;
    double h;     // spacing 2^l h
    double dinv;  // 1 / (2D + sigma h^2): the local solve's factor (host-computed)
    void* e;      // padded iterate of (Delta_h - sigma) e = rhs (final iterate of a V-cycle)
    void* rhs;    // right-hand side (same indexing as e)
    void* e2;     // 2D fused path: the pre-smoothed iterate (same indexing as e)
    void* rhs2;   // 2D level 0 only (else null): the right-hand side of odd outer steps
};

// Right-hand side of level `level` during outer step `it`.  Level 0 of a 2D instance with
// fused levels keeps two buffers, so that the kernel forming r_{N+1} never writes the
// array other tiles are still reading r_N from: step N uses rhs for even N, rhs2 for odd.
__host__ __device__ inline void* lev_rhs(const LevelDesc& L, int level, int it)
{
    return (level == 0 && L.rhs2 && (it & 1)) ? L.rhs2 : L.rhs;
}

struct InstDesc {
    int D, n, nlev, ltail;      // ltail: first level solved inside the one-CTA tail kernel
    int max_outer, nres_blocks; // residual tiles (one partial sum each)
    int res_tx, res_ty;         // residual tile grid (x tiles, y tiles); z tiles = n (3D)
    double h, k2, tol;
    double ih2, cdiag;          // 1/h^2 and k^2 - 2D/h^2 (the stencil's diagonal)
    double sigma;               // alpha - k^2 >= 0: inner operator Delta_h - sigma
    double damp;                // p >= 0: damping term i p u of Delta u + (i p + k^2) u = f
    double2* u[2];              // u[0] = caller's array, u[1] = library buffer
    const double2* f;
    const double2* g;
    double* part;               // [2 * nres_blocks]: sum |r|^2 partials, then max |e|^2
    unsigned int* count;        // residual tiles finished in the current launch
    double* hist;               // relres_0..relres_max_outer
    double* einf;               // ||e_N||_inf, N = 0..max_outer-1
    LevelDesc lev[HELM_MAXLEV];
};

struct InstState {
    int status;      // HELM_ST_ACTIVE while iterating, else the outcome
    int it;          // outer steps performed (u_it lives in u[it & 1])
    int run;         // consecutive non-decreasing relres steps
    int pad_;
    double norm0;    // ||r_0||_2
    double prev;     // relres of the previous step
    double rmin;     // smallest relres so far
};

// Work item of a multigrid launch: one (instance, level) pair; blocks stride over it.
struct MgItem {
    int inst;
    int level;
};

// Work item of a residual launch: one tile of one instance.
struct ResItem {
    int inst;
    int tx, ty, tz;
};

template <typename R> struct C2;
template <> struct C2<float>  { typedef float2  T; };
template <> struct C2<double> { typedef double2 T; };

__host__ __device__ inline int round_up(int a, int b) { return (a + b - 1) / b * b; }

// Slot of node x within an x-row of a level array: x itself in 2D, the colour-split slot
// in 3D (even x at x/2, odd x at pitch/2 + x/2; pitch is a multiple of 16).
template <int D>
__host__ __device__ __forceinline__ int xslot(int x, int pitch)
{
    return (D == 3) ? ((x & 1) ? (pitch >> 1) + (x >> 1) : (x >> 1)) : x;
}

}  // namespace helm
