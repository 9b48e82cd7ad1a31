// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <string>
#include <utility>
#include <vector>

#include "ik.h"

namespace ikb {

// Offsets are packed as three signed bytes: x | y << 8 | z << 16.
__host__ __device__ inline int32_t pack3(int x, int y, int z) {
  return (int32_t)((uint32_t)(x & 0xff) | ((uint32_t)(y & 0xff) << 8) | ((uint32_t)(z & 0xff) << 16));
}
__host__ __device__ inline int unpack_x(int32_t v) { return (int)(int8_t)(v & 0xff); }
__host__ __device__ inline int unpack_y(int32_t v) { return (int)(int8_t)((v >> 8) & 0xff); }
__host__ __device__ inline int unpack_z(int32_t v) { return (int)(int8_t)((v >> 16) & 0xff); }

struct Dims {
  int nx, ny, nz;  // voxels
  int wx;          // words per row = nx / 32
  long nw;         // words per set
};

// One admissible-offset table on the host, built by tables.cpp.
struct ShellHost {
  int lo2 = 0, hi2 = 0;
  std::vector<int32_t> off;       // packed offsets, ordered by (|d|^2, z, y, x)
  // device order: offsets sorted by (z, y, x), so that the offsets of one
  // (dz, dy) row are contiguous; rows[(dz+R)*(2R+1) + (dy+R)] .. rows[.. + 1]
  // is the range of row (dy, dz).
  int R = 0;
  std::vector<int32_t> dev_off;
  std::vector<int32_t> rows;      // size (2R+1)^2 + 1
  std::vector<int32_t> sc_start;  // size n + 1, into sc, device order
  std::vector<int32_t> sc;        // packed supercover voxels of 0 -> dev_off[i], (z, y, x) order
  int max_sc = 0;
};

void shell_bounds(int len, double tol, int* lo2, int* hi2);
// Approach cone on a segment: offset s is kept when s.a > 0 and
// den * (s.a)^2 >= num * |s|^2 * |a|^2 (cos^2 of the half-angle = num / den).
struct ConeSpec {
  int ax, ay, az, num, den;
};
// The shell lo2 <= |d|^2 <= hi2, or its part inside `cone` when given (R
// stays floor(sqrt(hi2)), the reach of the whole shell).
void build_shell(int lo2, int hi2, ShellHost* out, const ConeSpec* cone = nullptr);
// The row-lane table of a shell (SegDev::tabr, rowsr); empty for reach > 31.
void build_row_table(const ShellHost& h, std::vector<int32_t>* tabr, std::vector<int32_t>* rowsr);
// The row-lane edge masks' supercover table (ShellDev::d_sctabr); empty for reach > 31.
void build_row_mask_table(const ShellHost& h, std::vector<int32_t>* sctabr);
// Closed supercover of 0 -> d by incremental traversal; (z, y, x) order.
void supercover_traverse(int dx, int dy, int dz, std::vector<int32_t>* out);
// The same walk into a caller buffer of cap entries, allocating nothing:
// returns the number of voxels, or -1 when they do not fit.
int supercover_walk(int dx, int dy, int dz, int32_t* out, int cap);

// A box of words {wx0..wx1} x {y0..y1} x {z0..z1} (inclusive) over which
// edge masks are stored; a mask row holds its words in (z, y, x) order.
struct MaskBox {
  int wx0, y0, z0, wx1, y1, z1;
  __host__ __device__ int nwx() const { return wx1 - wx0 + 1; }
  __host__ __device__ int nyy() const { return y1 - y0 + 1; }
  __host__ __device__ long words() const { return (long)nwx() * nyy() * (z1 - z0 + 1); }
  __host__ __device__ long index(int wx, int y, int z) const {
    return ((long)(z - z0) * nyy() + (y - y0)) * nwx() + (wx - wx0);
  }
  __host__ __device__ bool contains(const MaskBox& o) const {
    return o.wx0 >= wx0 && o.wx1 <= wx1 && o.y0 >= y0 && o.y1 <= y1 && o.z0 >= z0 && o.z1 <= z1;
  }
};

// Device view of one segment's tables.
struct SegDev {
  const int32_t* off;      // [n] packed offsets, device order (z, y, x)
  const int32_t* rows;     // [(2R+1)^2 + 1] row starts, see ShellHost
  const int32_t* sc_start; // [n + 1]
  const int32_t* sc;       // packed supercover voxels
  const uint32_t* mask;    // [n][box words] edge masks over the word box `mbox`: bit of voxel p
                           // in row e = segment p -> p + off[e] free; nullptr: each test walks
                           // the supercover against occ
  MaskBox mbox;            // words of the grid the masks cover (every word a test can read)
  int n;
  int lo2, hi2;
  int R;                   // max |component| of an offset
  const int32_t* tab;      // [n] shared-memory deltas for the tiled kernel, see TileCfg
  const int32_t* tabw;     // [n] the same for rows staged without pad words (pitch wx):
                           // ((dy * wx + (dx >> 5)) << 6) | (dx < 0) << 5 | (dx & 31); nullable
  const int32_t* tabr;     // [n] the row-lane propagation's offsets: per dz plane those with dx < 0
                           // ordered by (dy, dx), then those with dx >= 0; entry
                           // (e << 11) | ((dy + 32) << 5) | (dx & 31), e the offset's index
                           // above (its edge-mask row); nullable (reach above 31)
  const int32_t* rowsr;    // [(2R+1) * 2 * (2R+2)] run starts of tabr: (dz, sign, dy), each
                           // (dz, sign) run ending at its entry dy = R + 1
  const int32_t* sctab;    // [sc_start[n]] shared-memory deltas of the supercover voxels
  const uint32_t* occ;     // the grid's occupancy, for segment tests without stored masks
};

// Output tiling of the shared-memory propagation kernel: a block of 8 warps
// covers all wx words of TY rows in each of TZ = 8 z slices (warp i = slice
// z0 + i, lane = (word lane % wx, row lane / wx)); its source halo of reach R
// is staged in shared memory as (TZ + 2R) x (TY + 2R) rows of P words (word
// -1 .. wx, zero-padded), P the narrowest pitch with at most 2-way bank
// conflicts among a warp's row-word addresses.  tab[e] = ((dy * P + (dx >> 5)) << 5) | (dx & 31): the
// shared-memory word delta and the funnel shift of offset e.
struct TileCfg {
  int TY, TZ, P, lanes, tiles_y, tiles_z;
  int depth = 8;  // output slices per tile of the propagation: 8 (one per warp) or 16 (two)
  int pair = 1;   // IK_OPT_QUERY_PAIRS: 0 one query per block, 1 two (padded rows), 2 two (rows without pad)
  int rows = 1;   // IK_OPT_ROW_LANES: the row-lane propagation where it applies
};
TileCfg make_tile_cfg(const Dims& d);
// Shared-memory bytes of the tiled kernel for reach R (0 if it does not apply).
size_t tile_smem_bytes(const TileCfg& tc, int R);
// Both halos (X and occupancy) of the tiled propagation without stored edge
// masks; 0 when they do not fit in kTileOccSmemMax bytes (the 227 KiB a block
// may opt in to, less 1 KiB for the kernel's static shared memory).
constexpr int kTileOccSmemMax = 226 * 1024;
size_t tile_occ_smem_bytes(const TileCfg& tc, int R);

// Bounding box of a voxel set in word coordinates, kept in "min form" so
// that every component accumulates with atomicMin: {wx0, y0, z0, -wx1, -y1,
// -z1}.  A box whose bytes are all 0x7f is empty (wx0 > wx1).
constexpr int kBoxEmptyByte = 0x7f;

// seg[k]: segment k+1's offsets as segment vectors s = p_{k+1} - p_k (the
// backward sets, tracebacks and validation read them so); segf[k]: the same
// segment mirrored, -s (the forward gathers read it so: joint k+1 at p takes
// its source at p - s).  A whole shell is symmetric, so both are the same
// table; a direction limit (a cone) makes them two.
struct ArmDev {
  SegDev seg[IK_MAX_SEG];
  SegDev segf[IK_MAX_SEG];
  int S;
  int len[IK_MAX_SEG];
};

// Device-resident shell table with its edge masks for one occupancy version.
struct ShellDev {
  ShellHost host;
  int32_t* d_off = nullptr;
  int32_t* d_rows = nullptr;
  int32_t* d_tab = nullptr;
  int32_t* d_sctab = nullptr;  // per supercover voxel: (shared-memory delta << 5) | (dx & 31)
  int32_t* d_sctab_tma = nullptr;  // the same for the TMA-staged brick (pitch tma_mask_pitch)
  int32_t* d_tabw = nullptr;       // SegDev::tabw (grids whose rows fill a warp: wx = 1, 2, 4, 8, 16, 32)
  int32_t* d_tabr = nullptr;       // SegDev::tabr, rowsr (reach at most 31)
  int32_t* d_rowsr = nullptr;
  int32_t* d_sctabr = nullptr;     // per supercover voxel, for the row-lane edge masks (reach at most 31):
                                   // ((vz * (32 + 2R) + vy) << 6) | (vx + 32)
  int32_t* d_sc_start = nullptr;
  int32_t* d_sc = nullptr;
  uint32_t* d_mask = nullptr;
  size_t mask_bytes = 0;         // allocated bytes of d_mask
  MaskBox mbox{0, 0, 0, -1, -1, -1};  // words covered by d_mask
  uint64_t mask_version = ~0ull;  // occupancy version the masks were built for
  int reach = 0;
};

// ------------------------------------------------------------- launchers
// All launchers enqueue on `st` and return the launch error (cudaSuccess).
cudaError_t launch_rasterize(const Dims& d, const int32_t* boxes, int n_boxes, uint32_t* occ,
                             cudaStream_t st);
// dst = src dilated by the ball |v|^2 <= r2 (src != dst).
cudaError_t launch_dilate(const Dims& d, const uint32_t* src, int r2, uint32_t* dst, cudaStream_t st);
// Edge masks of shell s over the word box b (mask rows of b.words() words).
cudaError_t launch_edge_masks(const Dims& d, const TileCfg& tc, const uint32_t* occ, const ShellDev& s,
                              const MaskBox& b, uint32_t* mask, cudaStream_t st);
// The same with the occupancy brick of every tile staged by a TMA tensor
// load: tmap is a CUtensorMap over occ (uint32 words, dims {wx, ny, nz}, box
// {BX, TY + 2R, TZ + 2R}, out-of-bounds fill zero) for BX = tma_mask_pitch(d)
// (0: the grid's rows are not 16-byte multiples, no TMA form); *slow counts
// blocks whose copy did not complete in time (they staged with loads).
int tma_mask_pitch(const Dims& d);
size_t tma_mask_smem_bytes(const TileCfg& tc, int R, int BX);
cudaError_t launch_edge_masks_tma(const Dims& d, const TileCfg& tc, const void* tmap, const uint32_t* occ,
                                  const ShellDev& s, const MaskBox& b, uint32_t* mask, int* slow,
                                  cudaStream_t st);
// out[q] = (mask ? mask[q] : ~0) & D_seg(X[q]) for q < Q; sets are nw words
// apart with stride `x_stride` / `out_stride` / `mask_stride` words between
// queries (mask_stride 0: one mask shared by all queries).
// xbox / obox: boxes of X[q] and out[q] at q * box_stride ints; obox must
// be set empty beforehand and receives the box of the output.
// The tiled shared-memory kernel runs when tile_smem_bytes(tc, seg.R) > 0
// (for a segment without stored edge masks, when tile_occ_smem_bytes > 0:
// its supercover walks then read an occupancy halo in shared memory), the
// global-load kernel otherwise.
// Device scratch for the work list of a batched propagation: items {query,
// tile} (cap entries, at least Q x tiles), count[0] = items, count[1] = the
// next item to take; blocks = the grid of resident blocks that walks the
// list.
struct WorkList {
  int2* items;
  int* count;
  long cap;
  int blocks;
};
// Whether launch_propagate walks the work list wl (Q >= kListMinQueries on
// the tiled kernels of depth 8); when it does, launch_tile_list must have
// built the list on the same stream just before.
constexpr int kListMinQueries = 16;
bool propagate_listed(const TileCfg& tc, const SegDev& seg, int Q, long out_stride, const WorkList* wl);
// Zeroes the Q outputs and lists the (query, tile) pairs within reach R of
// X[q]'s box (xbox) and inside the output mask's box (mbox, one min-form box
// for all queries, nullable); only those are computed.
cudaError_t launch_tile_list(const Dims& d, const TileCfg& tc, int R, int Q, const int32_t* xbox,
                             long box_stride, const int32_t* mbox, uint32_t* out, long out_stride,
                             const WorkList& wl, cudaStream_t st);
cudaError_t launch_propagate(const Dims& d, const TileCfg& tc, const SegDev& seg, const uint32_t* X,
                             long x_stride, const uint32_t* mask, long mask_stride,
                             const uint32_t* occ, uint32_t* out, long out_stride, int Q,
                             const int32_t* xbox, int32_t* obox, long box_stride, cudaStream_t st,
                             unsigned long long* counters = nullptr, const WorkList* wl = nullptr);
// counters (nullable, 4 x u64, accumulated): offset-word pairs visited,
// pairs whose shifted input word is non-zero, edge-mask words read, output
// words with a non-empty mask.
// Single-voxel seeds: set q = {p_q} & (and_set ? and_set : all) & ~excl,
// p_q from points[q] (int32 x, y, z) -- a point outside the grid gives the
// empty set.  found_gate (nullable): query q is seeded only when
// found_gate[q] != 0.
// obox (set empty beforehand, stride box_stride) receives each seed's box.
cudaError_t launch_seed_points(const Dims& d, const int32_t* points, int Q, const uint32_t* and_set,
                               const uint32_t* excl, uint32_t* out, long out_stride,
                               const int32_t* found_gate, int32_t* obox, long box_stride,
                               cudaStream_t st);
cudaError_t launch_and(const uint32_t* a, const uint32_t* b, uint32_t* out, long n, cudaStream_t st);
// Reach traceback over Q queries: V sets [Q][S+1][nw] (query stride vstride).
cudaError_t launch_traceback(const Dims& d, const ArmDev& arm, const int32_t* root,
                             const uint32_t* V, long vstride, int Q, int32_t* poses,
                             int32_t* found, cudaStream_t st);
// Replan re-solve: like traceback but minimising squared distance to
// old_pose first (old_pose [S+1][3]).
cudaError_t launch_traceback_nearest(const Dims& d, const ArmDev& arm, const int32_t* root,
                                     const uint32_t* V, const int32_t* old_pose, int32_t* pose,
                                     int32_t* found, cudaStream_t st);
// Guide points + waypoint target seeds for P paths of W waypoints:
// reach [P][S+1][3], found [P] (nullable: all found), writes
// g [P][W][3], eps_used [P][W] and V_S^(p,j) = F_S & T_j into
// Vw + ((p*W + j) * (S+1) + S) * nw.  Waypoints j < j_lo are skipped.
// wbox: boxes [P][W][S+1][6]; the box of each seeded set (index S) is
// accumulated (set empty beforehand).
// The polyline the guide points follow: `reach` holds, per path, the S + 1
// joints of a pose of this arm (segment count and nominal lengths).
struct GuideArm {
  int S;                // segments of the guide polyline (joints 0 .. S of `reach`)
  int len[IK_MAX_SEG];  // their nominal lengths; len[S]: the folded segment's (fold_len > 0)
  int n_per_seg = 0;    // 0: W points by the nominal arc rule; n: n points per segment (W = S n + 1)
  int pose_joints = 0;  // joints per pose record of `reach` (0: S + 1)
  int fold_len = 0;     // > 0: also the fold points, for a last segment of this length
};
// Guide points and waypoint targets.  The guide follows `reach` with the
// arm `ga` (nullptr: the path's own arm); the targets are laid out for `arm`.
// fold_at (nullable, [P][W][4]): for ga->fold_len > 0, the point the folded
// last segment aims at from waypoint j, as {A_x, A_y, A_z, den} = A / den:
// nominal arc length fold_len beyond the guide point on the polyline of
// `reach` (joints 0 .. S + 1).
cudaError_t launch_guide_targets(const Dims& d, const ArmDev& arm, const uint32_t* occ,
                                 const uint32_t* F_S, const int32_t* reach, const int32_t* found,
                                 int P, int W, int j_lo, int eps2, int eps2_max, int32_t* g,
                                 int32_t* eps_used, uint32_t* Vw, int32_t* wbox, cudaStream_t st,
                                 const int32_t* c_arr = nullptr, const GuideArm* ga = nullptr,
                                 int32_t* fold_at = nullptr);
// Smooth chains for P paths (one block each).  mode 0 = plan (backward from
// the reach pose), mode 1 = forward from pose c (replan).  scratch: per path
// 2 * (S+1) * nw zeroed words.
struct ChainArgs {
  int P, W, c, mode;
  int delta, max_relax;
  const int32_t* found;     // [P] nullable
  const uint32_t* Vw;       // [P][W][S+1][nw]
  const int32_t* eps_used;  // [P][W]
  int32_t* poses;           // [P][W][S+1][3]; plan: pose W-1 preset; replan: poses 0..c preset
  int32_t* relax;           // [P][W][2]
  int32_t* status;          // [P]
  uint32_t* scratch;
  int relaxed_eps_base;     // eps2 requested (to flag eps growth)
  const int32_t* c_arr = nullptr;  // replan: per-path current waypoint (else c)
  // per_joint: joint k = 1..S moves at most rad[k] + m voxels at relaxation
  // m (rad[0] unused; -1: joint k is not filtered -- it stays in its
  // survivor set, searched over that set's box from vbox); otherwise every
  // joint moves at most delta + m
  bool per_joint = false;
  int rad[IK_MAX_SEG + 1];
  const int32_t* vbox = nullptr;  // [P][W][S+1][6] min-form word boxes of the survivor sets
  // nullable, accumulated: [0] (offset, word) pairs the restricted
  // propagations visited, [1] those whose shifted source word was non-zero
  unsigned long long* counters = nullptr;
};
cudaError_t launch_smooth_chain(const Dims& d, const ArmDev& arm, const ChainArgs& a,
                                cudaStream_t st);
// Poses [P][W][S+1][3] of a path whose follower is joint S - 1: joints
// 0 .. S-1 from tposes [P][W][S][3], the last segment folded towards the
// fold points [P][W][4] (see launch_guide_targets) with segment S's tables
// sg; a pose whose last segment has no free end records -1 in relax [P][W][2]
// and sets status [P] to IK_PATH_BROKEN.
cudaError_t launch_fold_last(const Dims& d, const SegDev& sg, int S, int P, int W, const int32_t* tposes,
                             const int32_t* fold_at, int32_t* poses, int32_t* relax, int32_t* status,
                             cudaStream_t st);
// p[0 .. n) = v.
cudaError_t launch_fill_i32(int32_t* p, long n, int32_t v, cudaStream_t st);
// Records a CUDA error's text for ik_last_error_message (this thread).
void note_cuda_error(cudaError_t e);
// Opt-in to large dynamic shared memory for the tiled kernels (current device).
cudaError_t set_kernel_attributes();
cudaError_t launch_traceback_nearest_many(const Dims& d, const ArmDev& arm, const int32_t* root,
                                          const uint32_t* V, long vstride, const int32_t* old_pose,
                                          long old_stride, int32_t* pose, int32_t* found,
                                          const int32_t* gate, int Q, cudaStream_t st);
// Batched replan bookkeeping (see ik_kernels.cu).
cudaError_t launch_replan_prepare(int R, int W, int S, const int32_t* poses_in, const int32_t* c,
                                  const int32_t* valid, int32_t* cut, int32_t* need, int32_t* tgt,
                                  int32_t* relax, cudaStream_t st);
cudaError_t launch_replan_fix(int R, int W, int S, const int32_t* poses_in, const int32_t* cut,
                              const int32_t* need, int32_t* reach, int32_t* rfound, int32_t* gate,
                              cudaStream_t st);
cudaError_t launch_replan_finalize(int R, int W, int S, const int32_t* c, const int32_t* cut,
                                   const int32_t* gate, int32_t* poses, int32_t* relax,
                                   int32_t* status, cudaStream_t st);
// out[w] = T[w] & F[w] (a target set within reach), with its word box.
cudaError_t launch_seed_set(const Dims& d, const uint32_t* T, const uint32_t* F, uint32_t* out,
                            int32_t* obox, cudaStream_t st);
cudaError_t launch_validate(const Dims& d, const ArmDev& arm, const uint32_t* occ,
                            const int32_t* poses, int n, int32_t* valid, cudaStream_t st);

// ------------------------------------------------ persistent uneven batch
// One resident-block launch solves a whole batch of independent reach +
// path problems (each with its own grid, arm, root, target and waypoint
// count).  A problem moves through stages -- rasterise (slabs of 16 z
// slices), forward seed, forward levels 1..S, reach seed, reach levels S..1,
// traceback, guide points (one item per waypoint), waypoint levels S..1
// (items per (tile, waypoint)), smooth chain -- and the block that finishes
// the last item of a stage pushes the next stage's items onto one device
// queue (the tiles within reach of the source sets' boxes), so no item waits
// on another.  Blocks wait only for a queue slot to be published, with a
// time limit after which the launch gives up and the unfinished problems
// report IK_ERR_TIMEOUT.
constexpr int kBatchThreads = 512;  // 16 warps: 16-slice tiles, and the chain's block size
constexpr int kBatchTZ = 16;
constexpr int kBatchSlab = 16;      // z slices per rasterise item

struct BatchProb {
  Dims d;
  TileCfg tcs[IK_MAX_SEG];  // tiling of the propagation of segment k+1
  ArmDev arm;
  int S, W, n_boxes, n_slabs;
  int root[3], target[3];
  const int32_t* boxes;  // [n_boxes][6], inclusive
  // the problem's own buffers (each 128-byte aligned, written before read)
  uint32_t *occ, *F, *V, *Vw, *chain;
  int32_t *Fbox, *Vbox, *Vwbox, *reach, *found, *g, *eps, *poses, *relax, *status;
  // the caller's packed outputs for this problem
  int32_t *o_found, *o_reach, *o_poses, *o_relax, *o_status, *o_rc;
};

struct BatchQueue {
  int4* items;  // {problem + 1 (0: slot not yet published), stage, a, b}
  long long cap;
  unsigned long long* ctl;  // [0] next slot to take, [1] slots reserved, [2] problems done,
                            // [3] items completed (progress), [4] error (1: timeout, 2: overflow)
  int2* state;              // per problem: {stage, items of the stage still pending}
};

struct BatchRules {
  int delta, eps2, eps2_max, max_relax;
};

// Dynamic shared memory the persistent kernel needs besides its tile halos.
size_t batch_chain_smem_bytes();
cudaError_t batch_set_smem(size_t bytes);
// The dynamic shared memory one block of the persistent kernel may take.
size_t batch_smem_limit();
cudaError_t launch_batch_persistent(const BatchProb* probs, int n, const BatchQueue& q, const BatchRules& r,
                                    int blocks, size_t smem, long long timeout_ns, cudaStream_t st);

}  // namespace ikb
