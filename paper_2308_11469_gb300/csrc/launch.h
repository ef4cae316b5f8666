// Host-side launchers of the library's kernels (one translation unit per kernel family).
// Every launcher enqueues on `s` and returns the cudaError_t of the launch.
#pragma once
#include <cuda_runtime.h>
#include "common.cuh"

namespace helm {

// Tail-level bounds: levels with n <= these are solved inside one CTA in shared memory.
constexpr int TAIL_N_2D = 63;
constexpr int TAIL_N_3D = 15;
// FP64 keeps fewer levels in the one-CTA tail: on GB300 the FP64 rate of a single SM is
// small, so FP64 coarse levels run faster spread over the GPU.
// Set the inner operator's shift sigma (= alpha - k^2) of a descriptor and every level's
// local-solve factor 1 / (2D + sigma h_l^2) (computed here once, in FP64, so that no
// kernel thread divides).
inline void set_shift(InstDesc& d, double sigma)
{
    d.sigma = sigma;
    for (int l = 0; l < d.nlev; ++l) d.lev[l].dinv = 1.0 / (2.0 * d.D + sigma * d.lev[l].h * d.lev[l].h);
}

inline int tail_top(int D, int prec_is_fp64)
{
    if (prec_is_fp64) return D == 2 ? 31 : 7;
    return D == 2 ? TAIL_N_2D : TAIL_N_3D;
}

// ---- multigrid (vcycle.cu); prec: 0 = double, 1 = float ----
// mode 0: plain half-sweep; modes 1/2: first half-sweep of a pre-smoothing whose
// iterate is known to be zero on levels > 0 (mode 1) or on every level (mode 2): it
// writes both colours (this colour from rhs alone, the other colour as zero).
// nmax: the largest level of the launch (0 if not known: the generic kernel)
cudaError_t launch_rbgs(int D, int prec, const InstDesc* insts, const InstState* st,
                        const MgItem* items, int nitems, int work, int color, int mode,
                        cudaStream_t s, int nmax = 0);
// coarse rhs := full weighting of (rhs - (Delta_h - sigma) e) on level l, coarse e := 0;
// mode 2 / 1 (no pre-smoothing): the iterate is zero on every level / levels > 0, the
// residual is rhs and the coarse iterate is left to the prolongation
cudaError_t launch_restrict(int D, int prec, const InstDesc* insts, const InstState* st,
                            const MgItem* items, int nitems, int work, cudaStream_t s, int mode = 0,
                            int nmax = 0);
// e_l += prolongation of e_{l+1}; mode 2 / 1: e_l := prolongation where e_l is zero;
// skip0: colour-0 nodes are left alone (a colour-0 half-sweep comes next)
cudaError_t launch_prolong(int D, int prec, const InstDesc* insts, const InstState* st,
                           const MgItem* items, int nitems, int work, cudaStream_t s, int mode = 0,
                           int skip0 = 0);
// zero the iterate of the listed levels (ring included)
cudaError_t launch_zero(int D, int prec, const InstDesc* insts, const InstState* st,
                        const MgItem* items, int nitems, int work, cudaStream_t s);
// tail.cu: one CTA per item runs V(nu1,nu2) on levels item.level..coarsest in shared
// memory; every item of one launch has top size n0.  load_e: start level 0 from its e in
// global memory instead of zero.
cudaError_t launch_tail(int D, int prec, int n0, const InstDesc* insts, const InstState* st,
                        const MgItem* items, int nitems, int nu1, int nu2, int load_e,
                        cudaStream_t s);
size_t tail_smem_bytes(int D, int prec, int n);
// size of the level the tail solves exactly instead of cycling (0: none); prec 0 = FP64
int tail_exact_n(int D, int prec);
// raise the tail kernel's dynamic shared-memory limit (once, before any capture)
cudaError_t setup_tail(int D, int prec);
// cluster tail (2D complex64, cycles without pre-smoothing, level 255 below the top): one
// 8-CTA cluster per item runs levels 255 (the item's level), 127, 63 and the exact level 31
// and writes level 255's iterate; nu2 in {1, 2}.  ctail_setup() sets its attributes once and
// returns how many of its clusters can be resident at once (0: none fits).
int ctail_setup();
cudaError_t launch_ctail(const InstDesc* insts, const InstState* st, const MgItem* items, int nitems,
                         int nu2, cudaStream_t s);
// shared-memory carve-out preferences of the generic and outer kernels
cudaError_t setup_generic(int D, int prec);
cudaError_t setup_outer();

// ---- fused 2D multigrid (vcycle2d.cu): two launches per level ----
// descent: nu1 sweeps + residual + restriction; e (or zero) -> e2, coarse rhs.
// zero_mode: 2 = every level's iterate is zero, 1 = levels > 0 are zero, 0 = load e.
// nmax: the largest level of the launch; with nu1 = 0 and zero_mode = 2 (every iterate
// zero) the descent is the restriction of rhs alone (k_restrict_rhs2d)
cudaError_t launch_down2d(int prec, const InstDesc* insts, const InstState* st, const MgItem* items,
                          int nitems, int max_tiles, int nu1, int zero_mode, int shape,
                          cudaStream_t s,
                          int nmax = 0);
// ascent: e2 + prolongation of the coarse e, nu2 sweeps -> e
// e2_mode: 0 = read e2; 2 = e2 is zero on every level, 1 = below the finest level (no
// pre-smoothing from a zero iterate: the descent did not write it)
cudaError_t launch_up2d(int prec, const InstDesc* insts, const InstState* st, const MgItem* items,
                        int nitems, int max_tiles, int nu2, int shape, int e2_mode, cudaStream_t s);
// tile shape of a level (0 = 64 x 32, 1 = 32 x 16 for n <= 511) and its tile count
int tile_shape2d(int n);
int tiles2d(int n);
int tiles2d_for(int n, int shape);
// two descent steps of cycles without pre-smoothing from a zero iterate in one launch:
// every item (instance, level l) gets level l+1's and level l+2's rhs by full weighting;
// nmax: the largest level l of the launch
cudaError_t launch_restrict2_2d(int prec, const InstDesc* insts, const InstState* st, const MgItem* items,
                                int nitems, int nmax, cudaStream_t s);
cudaError_t setup_2d(int prec);

// ---- outer FP64 iteration (outer.cu) ----
// mode 0: r_0 from u[it&1]; mode 1: u[(it+1)&1] = u[it&1] + e_0, then r from it.
// Writes r into level-0 rhs (inner precision) and per-tile partials; the last tile of
// each instance forms relres, records the history and applies the status rule.
// ctrl != nullptr folds the step control (k_check) into the launch: the last of the
// launch's `ninst` instances to finish its residual scans `nscan` statuses, counts the
// step and sets the WHILE node's condition (use_cond).  damp != 0: some instance has a
// damping term p (the kernel variant that forms it).
cudaError_t launch_residual(int D, int prec, const InstDesc* insts, InstState* st,
                            const ResItem* items, int nitems, int mode, cudaStream_t s,
                            int* ctrl = nullptr, int nscan = 0, int ninst = 0, int use_cond = 0,
                            unsigned long long cond_handle = 0, int damp = 0);
// 2D, complex64 inner solves: level 0's ascent (launch_up2d with nu2 sweeps, e2_mode)
// fused with the mode-1 residual launch and its folded step control (same arguments as
// launch_residual's).  items: the level-0 items of every instance (all of size n), whose
// level 0 keeps two right-hand-side buffers.  Level 0's e is not written.
// l1f: level 1's ascent (prolongation from level 2 + nu2 sweeps, its iterate zero before, no
// pre-smoothing) is formed inside each tile on the coarse window it reads, in place of
// level 1's own ascent launch (every instance: level 1 a fused level, its e2 zero).
cudaError_t launch_upres2d(const InstDesc* insts, InstState* st, const MgItem* items, int nitems, int n,
                           int nu2, int e2_mode, cudaStream_t s, int* ctrl, int nscan, int ninst,
                           int use_cond, unsigned long long cond_handle, int damp, int l1f = 0);
int upres2d_tiles(int n);
int residual_tile_rows(int D);
int residual_tile_planes(int D);
int residual_tile_cols(int D);
// Any instance still iterating?  Counts the step, sets the while-loop condition.
cudaError_t launch_check(const InstState* st, int ninst, int* ctrl, int use_cond,
                         unsigned long long cond_handle, cudaStream_t s);
// constant fill of a complex128 array; max Re over a padded array's interior (>= 0)
cudaError_t launch_fill_c128(void* p, long count, double re, double im, cudaStream_t s);
cudaError_t launch_max_re(int D, int n, const void* u, unsigned long long* out, cudaStream_t s);
// power iteration on the finest level of instance 0 (interior nodes): fill e (which = 0)
// or rhs (1) with a real constant; out = sum |e|^2 (partial: power_iteration_blocks()
// doubles); rhs = sc * e
cudaError_t launch_lev_fill(int D, int prec, const InstDesc* insts, int which, double value, cudaStream_t s);
cudaError_t launch_lev_sumsq(int D, int prec, const InstDesc* insts, double* partial, double* out,
                             cudaStream_t s);
cudaError_t launch_lev_scale(int D, int prec, const InstDesc* insts, double sc, cudaStream_t s);
int power_iteration_blocks();
cudaError_t run_fp_bits_check(int count, unsigned long long seed, unsigned long long* bad_host);
// FP64 FMA rate of the current device (independent chains on every SM), best of 5 timed
// launches: TFLOP/s (an FMA counts 2 flops) and that launch's milliseconds
cudaError_t run_fp64_rate(double* tflops, double* ms_best);
// the residual tile list of one instance: item q = (instance 0, q mod tx, (q / tx) mod ty,
// q / (tx ty)), the order the host loops would give (x fastest)
cudaError_t launch_fill_res_items(ResItem* items, int tx, int ty, int tz, cudaStream_t s);
// A new instance's workspace set-up: ws[0, bytes) zeroed (ws 16-byte aligned) and its
// residual tile list (tx x ty x tz tiles, instance 0) written at items.  One launch sets up
// `count` instances from a device array of these records.
struct WsInit {
    unsigned char* ws;
    unsigned long long bytes;
    ResItem* items;
    int tx, ty, tz, pad;
};
cudaError_t launch_init_workspaces(const WsInit* recs, int count, cudaStream_t s);
// u[0] and u[1] rings := g ring
cudaError_t launch_set_ring(int D, const InstDesc* insts, int inst, int n, cudaStream_t s);
// the same for the m instances insts[slots[j]] (device list), all of size n
cudaError_t launch_set_ring_many(int D, const InstDesc* insts, const int* slots, int m, int n, cudaStream_t s);
// the residual tiles (tx x ty x tz each) of instances slots[0 .. m) into items, in order
cudaError_t launch_fill_res_many(ResItem* items, const int* slots, int m, int tx, int ty, int tz, cudaStream_t s);
// interior tight <-> level-0 padded/pitched, inner precision
cudaError_t launch_pack(int D, int prec, const InstDesc* insts, int inst, int n,
                        const void* src, int which /*0 = e, 1 = rhs*/, cudaStream_t s);
cudaError_t launch_unpack(int D, int prec, const InstDesc* insts, int inst, int n,
                          void* dst, cudaStream_t s);

// error text of the last failing call (helm_last_error), launch counter (helm_launch_count),
// device-pointer check of the C ABI (non-null, 16-byte aligned, device or managed memory)
void note_error(const char* msg);
void add_launches(uint64_t n);
bool device_pointer_ok(const void* p);

}  // namespace helm
