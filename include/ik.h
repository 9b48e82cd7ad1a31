/*
 * ik.h -- C ABI of the B300 gap map-seeking inverse-kinematics library.
 *
 * The library solves the problem stated in the paper's Introduction (eq 1):
 * find a chain of segment translations that takes the arm root p_root to the
 * end-effector target p_end, among obstacles, then a smooth sequence of poses
 * along the way (section "Path Planning") and, when obstacles move, a new
 * remainder of that sequence (section "Dynamic Obstacles").
 *
 * Lattice form used throughout (the paper's quiver and n-point collision
 * test restated exactly on the voxel grid):
 *   - the grid is nx * ny * nz unit voxels, nx a multiple of 32; a voxel set
 *     is a bit-packed array of uint32 words, x fastest: voxel (x, y, z) is bit
 *     (x % 32) of word (z * ny + y) * (nx / 32) + x / 32;
 *   - occupancy uses 1 = occupied (the paper's mask, section "The
 *     representations of the arm and obstacles", stores 0 for obstacles; the
 *     meaning is the same);
 *   - segment k of nominal length L_k may take any integer offset d with
 *     lo2 <= |d|^2 <= hi2, lo2 = max(1, ceil((L_k - tol)^2)),
 *     hi2 = floor((L_k + tol)^2), evaluated in double precision ("shell";
 *     stands in for the quiver of section "Discretization of the segment
 *     articulations" and the epsilon on the gap vector of "The gap in gMS");
 *   - a segment p->q is obstacle-free when every voxel whose closed unit cube
 *     meets the closed segment is free (closed supercover; stands in for the
 *     n sample points of "Testing for collisions");
 *   - a pose is int32 [n_seg + 1][3] joint positions (x, y, z), p_0 = root.
 *
 * Conventions for every call:
 *   - return value: IK_OK (0) or a negative IK_ERR_* code; nothing throws
 *     across the ABI; "no solution" is not an error (found = 0, or a path
 *     status);
 *   - ownership: the caller owns every buffer it passes; the library owns the
 *     grid's device state (occupancy, shell tables, edge masks, reachable
 *     sets, scratch) from ik_create_grid until ik_destroy_grid;
 *   - pointers are host pointers unless a call takes an `on_device` flag and
 *     it is non-zero, in which case the listed arrays are device pointers of
 *     the grid's device;
 *   - calls are synchronous on the grid's CUDA stream; a handle must not be
 *     used from two threads at once;
 *   - on a GPU fault or a failed allocation the call returns IK_ERR_CUDA or
 *     IK_ERR_OOM; ik_last_error_message() gives the CUDA error text.
 */
#ifndef IK_B300_H
#define IK_B300_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define IK_API __attribute__((visibility("default")))
#else
#define IK_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ----------------------------------------------------------- return codes */
#define IK_OK 0
#define IK_ERR_ARG -1         /* invalid argument (sizes, coordinates, NULL) */
#define IK_ERR_OOM -2         /* device or host allocation failed */
#define IK_ERR_CUDA -3        /* a CUDA call failed */
#define IK_ERR_TIMEOUT -4     /* a bounded device-side wait ran out */
#define IK_ERR_STATE -5       /* call made in the wrong state (e.g. no obstacles set) */
#define IK_ERR_UNSUPPORTED -6 /* valid request beyond this build's limits */

/* ------------------------------------------------------------ path status */
#define IK_PATH_OK 0          /* every waypoint solved with the nominal filter */
#define IK_PATH_RELAXED 1     /* some waypoint needed a wider filter or target ball */
#define IK_PATH_BROKEN 2      /* some waypoint had no solution; it repeats its neighbour */
#define IK_PATH_UNREACHABLE 3 /* no reach pose exists (or the given one is invalid) */
#define IK_PATH_KEPT 4        /* replan: the remainder is still valid and unchanged */

typedef struct ik_grid_s* ik_grid;

/* An arm: n_seg segments (1..IK_MAX_SEG) of integer nominal lengths
 * len[k] >= 1 voxels (k = 0 is the segment at the root), and the shell
 * tolerance tol (0.5 by default: the shell of L is then exactly
 * L^2 - L + 1 <= |d|^2 <= L^2 + L). */
#define IK_MAX_SEG 16
#define IK_MAX_LEN 100
typedef struct {
  int32_t n_seg;
  const int32_t* len;
  float tol;
} ik_arm;

/* Path parameters (sections "Smooth sequence computation", "Filtering for
 * smoothness"):
 *   n_way      number of waypoints W >= 2; waypoint 0 is the root, W-1 the target;
 *   delta      each joint moves at most delta voxels (Euclidean) between
 *              consecutive poses; on failure at a waypoint the bound grows by
 *              one voxel at a time, only after a failure;
 *   eps2       the end effector lands within squared distance eps2 of the
 *              waypoint (a looser tolerance than the reach's); if no free voxel is that close
 *              the radius grows by one unit of eps2 up to eps2_max;
 *   max_relax  cap on the number of delta increments, -1 = until the ball
 *              covers the grid. */
typedef struct {
  int32_t n_way;
  int32_t delta;
  int32_t eps2;
  int32_t eps2_max;
  int32_t max_relax;
} ik_path_params;

/* ---------------------------------------------------------- housekeeping */
IK_API int ik_version(void);
IK_API const char* ik_strerror(int code);
/* Text of the last CUDA error seen by this process ("" if none). */
IK_API const char* ik_last_error_message(void);

/* Create a grid on the current CUDA device.  nx % 32 == 0, each extent in
 * [32, 1024] for nx and [1, 1024] for ny, nz.  cuda_stream may be NULL (the
 * legacy default stream).  The occupancy starts all free. */
IK_API int ik_create_grid(int nx, int ny, int nz, void* cuda_stream, ik_grid* out);
IK_API int ik_destroy_grid(ik_grid g);
/* Grid options.  IK_OPT_EDGE_MASKS (default 1): keep one edge mask per shell
 * offset and word (the segment test becomes one 4-byte read), over the words
 * the segment's joints can reach from the root (1.7 GB for the 128^3 grid
 * and the arm {20,18,...,6}); rebuilt when the occupancy changes.  With 0
 * every segment test walks the offset's supercover against the occupancy
 * instead: no mask memory and no rebuild, slower tests -- the better choice
 * for grids solved once.  Results are identical either way. */
#define IK_OPT_EDGE_MASKS 1
/* IK_OPT_TILE_DEPTH: output slices per block of the propagation kernel, 8
 * (one per warp) or 16 (two per warp, default 8).  Results are identical. */
#define IK_OPT_TILE_DEPTH 2
/* IK_OPT_DILATE_R2 (default 0 = off, at most 100): obstacles are dilated by
 * the ball |v|^2 <= value before anything uses them (section "Testing for
 * collisions": the obstacle volumes are dilated when the grid is set up, to
 * account for the arm's thickness and a clearance margin).  It applies to
 * the current occupancy at once and to every later ik_set_obstacles /
 * ik_set_boxes and to batches captured afterwards (a batch keeps the value it
 * was captured with); ik_get_obstacles returns the dilated occupancy. */
#define IK_OPT_DILATE_R2 3
/* IK_OPT_WORK_LIST: how a batched backward pass (16 or more queries) visits
 * the tiles of each level.  1 (default): a work list of the tiles a level's
 * bounding boxes reach, walked by a grid of resident blocks, on the levels
 * where a bound from the arm's reaches leaves at most an eighth of the tiles
 * (a sixteenth where the row-lane kernel runs the other levels), and one
 * block per (tile, query) elsewhere; 0: one block per (tile, query)
 * on every level; 2: the work list on every level.  Results are identical. */
#define IK_OPT_WORK_LIST 4
/* IK_OPT_QUERY_PAIRS: on the levels of a batched backward pass that run one
 * block per tile (not the work list), with stored edge masks, a block
 * carries two queries, which share the output mask and the edge-mask words:
 * 1 (default) with padded source rows; 2 with source rows staged without
 * pad words where a warp covers whole rows (conflict-free shared loads, the
 * bits read across a row's end masked per offset: measured slower on the
 * 128^3 step, 83.8 vs 79.1 ms, the masks cost more issue than the conflicts
 * did), else as 1; 0: one query per block.  Results are identical. */
#define IK_OPT_QUERY_PAIRS 5
/* IK_OPT_TMA_MASKS: 1: the edge-mask kernel stages each tile's occupancy
 * brick with one TMA tensor copy where the grid allows it (rows a multiple of
 * 16 bytes, nx a multiple of 128) and the brick fits in shared memory; 0
 * (default): per-thread loads.  The copy must start on a 16-byte boundary,
 * so a staged row is 12 words wide on a 128-voxel row instead of 6, which
 * halves the blocks per SM: on one B300 a rebuild of the 128^3 workload's
 * masks takes 6.77 ms with it and 5.81 ms without (256^3: 16.3 / 13.9 ms).
 * Results are identical. */
#define IK_OPT_TMA_MASKS 6
/* IK_OPT_ROW_LANES (default 1): the edge masks of shells of reach at most
 * 31 are built with a lane per row on grids whose rows are 1, 2, 4 or 8
 * words (nx = 32, 64, 128, 256; 5.78 -> 3.63 ms per 128^3 rebuild); and with
 * stored edge masks, on grids whose rows
 * are 1, 2 or 4 words (nx = 32, 64 or 128) and shells of reach at most 31,
 * the levels of a batched pass (two or more queries) that run one block per
 * tile (not the work list) use the row-lane kernel: a lane owns a whole
 * row (two queries' words where IK_OPT_QUERY_PAIRS allows), each offset's
 * source row comes from one conflict-free vector load of shared memory,
 * and the warps of a block take planes of offsets (dz) one at a time, each
 * packing the rows that can still gain bits (and whose source rows hold a
 * word) into full passes.  On one B300 the 128^3 reach + path step takes
 * 52.7 ms with it and 78.5 ms without.  0: the forms above.  Results are
 * identical. */
#define IK_OPT_ROW_LANES 7
IK_API int ik_set_option(ik_grid g, int option, int value);
/* Number of uint32 words of one voxel set of this grid. */
IK_API size_t ik_grid_words(ik_grid g);

/* ---------------------------------------------------------- obstacles */
/* Replace the occupancy with a bit-packed set (1 = occupied), n_words =
 * ik_grid_words(g).  Bits of x >= nx do not exist (nx % 32 == 0). */
IK_API int ik_set_obstacles(ik_grid g, const uint32_t* occ_words, size_t n_words, int on_device);
/* Replace the occupancy with the union of n_boxes inclusive boxes
 * boxes[i] = {lo_x, lo_y, lo_z, hi_x, hi_y, hi_z}, clipped to the grid (empty
 * boxes are allowed).  The boxes are rasterised on the GPU. */
IK_API int ik_set_boxes(ik_grid g, const int32_t* boxes, int n_boxes, int on_device);
IK_API int ik_get_obstacles(ik_grid g, uint32_t* occ_words, size_t n_words, int on_device);

/* ----------------------------------------------------------- reach IK */
/* Forward reachable sets F_0..F_S (section "The procedure for IK solution",
 * Steps 1 and 2A): F_0 = {root} if free, F_k = every voxel reachable from
 * F_{k-1} by an admissible obstacle-free segment k.  fsets_out is
 * [n_seg + 1][ik_grid_words(g)].  F is cached per (occupancy, root, arm). */
IK_API int ik_forward_sets(ik_grid g, const ik_arm* arm, const int32_t root[3], uint32_t* fsets_out,
                    int on_device);

/* Reach pose for one target (Steps 1, 2A, 2B and 3): the survivor sets
 * V_k = F_k & B_k (joint-k positions on some valid chain root -> target,
 * B_k the backward sets from the target) and the chosen pose: p_0 = root,
 * p_k = the voxel of V_k with the smallest linear index reachable from
 * p_{k-1} by a valid segment.  pose_out [n_seg + 1][3]; vsets_out nullable,
 * [n_seg + 1][words]; *found = 1 when a pose exists.  Root and target must be
 * inside the grid (else IK_ERR_ARG); an occupied root or target gives
 * found = 0. */
IK_API int ik_solve_reach(ik_grid g, const ik_arm* arm, const int32_t root[3], const int32_t target[3],
                   int32_t* pose_out, uint32_t* vsets_out, int* found);

/* The same for n targets sharing one root, solved together in batched
 * launches (one backward launch per segment for all targets).  targets
 * [n][3]; poses_out [n][n_seg + 1][3]; found_out [n]; vsets_out nullable
 * [n][n_seg + 1][words].  With on_device != 0 all four arrays are device
 * pointers. */
IK_API int ik_solve_reach_many(ik_grid g, const ik_arm* arm, const int32_t root[3],
                        const int32_t* targets, int n, int32_t* poses_out, int32_t* found_out,
                        uint32_t* vsets_out, int on_device);

/* ------------------------------------------- target cones and clouds */
/* Approach cone on the last segment (section "The gap in gMS": the backward
 * search from the target starts from the directions the last segment may
 * arrive along, one vector or a cone of them).  The segment vector s (from
 * joint n_seg - 1 to the end effector) is admissible when s . axis > 0 and
 * cos2_den * (s . axis)^2 >= cos2_num * |s|^2 * |axis|^2, i.e. its angle to
 * the axis is at most theta with cos^2 theta = cos2_num / cos2_den (exact
 * integer test).  axis != 0 with components in [-1024, 1024];
 * 0 <= cos2_num <= cos2_den <= 1000000, cos2_den >= 1 (else IK_ERR_ARG); a
 * cone that keeps no offset of the last segment's shell is IK_ERR_ARG. */
typedef struct {
  int32_t axis[3];
  int32_t cos2_num, cos2_den;
} ik_cone;

/* ik_solve_reach_many with the last segment restricted to `cone` (nullable:
 * no restriction, identical to ik_solve_reach_many).  The forward sets use
 * the whole shells; the backward sets from each target and the traceback
 * use the cone's offsets for the last segment, so a found pose ends at the
 * target with its last segment in the cone.  V_n_seg stays F_n_seg & {target}.
 * Arrays and on_device as for ik_solve_reach_many. */
IK_API int ik_solve_reach_many_cone(ik_grid g, const ik_arm* arm, const ik_cone* cone,
                                    const int32_t root[3], const int32_t* targets, int n,
                                    int32_t* poses_out, int32_t* found_out, uint32_t* vsets_out,
                                    int on_device);

/* Reach for a target set T (a cloud of targets, section "Dynamic
 * Obstacles"; host bit set of ik_grid_words(g) words, same layout as the
 * occupancy) with an optional approach cone.  V_n_seg = F_n_seg & T; the
 * chosen pose is the minimum-index traceback of the survivor sets, so its end
 * effector is the smallest-index voxel of T that the chain can reach.
 * pose_out [n_seg + 1][3]; vsets_out nullable [n_seg + 1][words]; *found. */
IK_API int ik_solve_reach_set(ik_grid g, const ik_arm* arm, const ik_cone* cone, const int32_t root[3],
                              const uint32_t* target_words, int32_t* pose_out, uint32_t* vsets_out,
                              int* found);

/* Per-segment direction limits (section "The procedure for IK solution",
 * Step 1 (a): joint 1 angle constraints -- section "The gap in gMS" gives the
 * first segment restricted to the upper hemisphere of the quiver, or less).
 * limits[k] restricts segment k+1's vector s = p_{k+1} - p_k to the cone of
 * ik_cone (same test and ranges as above); an all-zero axis leaves that
 * segment free; limits = NULL clears the arm's limits.  The limits belong to
 * the grid and to this arm (same lengths and tol) and apply to every later
 * call with it: forward sets, reach, waypoint sets, paths, replans,
 * validation and batches captured afterwards.  A limit that keeps no offset
 * of its shell makes those calls fail with IK_ERR_ARG; so does an approach
 * cone (ik_solve_reach_many_cone / ik_solve_reach_set) for an arm whose last
 * segment is limited.  The uneven batch (ik_solve_batch) and
 * ik_forward_sets_noalloc do not apply limits.  Only absolute directions are
 * expressible here: a limit on the angle between consecutive segments would
 * need the previous segment's direction in the state of the set propagation. */
IK_API int ik_set_segment_limits(ik_grid g, const ik_arm* arm, const ik_cone* limits);

/* --------------------------------------------------------------- path */
/* Guide waypoints on a reach pose (section "Path Planning"): W points spaced
 * evenly in nominal arc length Lambda = sum L_k along the polyline
 * p_0 .. p_S.  Waypoint j lies on segment k with
 * C_{k-1} <= j Lambda / (W-1) < C_k (C_k the cumulative nominal length; the
 * last waypoint on segment S) at fraction r / den,
 * r = j Lambda - C_{k-1} (W-1), den = L_k (W-1), rounded half up per
 * component: g_j = p_{k-1} + floor((2 r (p_k - p_{k-1}) + den) / (2 den)).
 * g_0 = root, g_{W-1} = end effector.  g_out [n_way][3]. */
IK_API int ik_guide(ik_grid g, const ik_arm* arm, const int32_t* reach_pose, int n_way, int32_t* g_out);

/* Survivor sets of every waypoint of one path in one batched pass (one
 * full IK per waypoint, section "Implementation Performance"):
 * T_j = free voxels within squared distance eps2 of g_j (grown up to
 * eps2_max when empty; T_{W-1} = {end effector of the reach pose}),
 * V^(j)_k = F_k & B^(j)_k.  eps2_used [n_way] (-1: no free voxel even at
 * eps2_max); vsets_out nullable [n_way][n_seg + 1][words]. */
IK_API int ik_waypoint_sets(ik_grid g, const ik_arm* arm, const int32_t* reach_pose, int n_way, int eps2,
                     int eps2_max, int32_t* eps2_used, uint32_t* vsets_out);

/* Smooth path to a reach pose (sections "Smooth sequence computation" and
 * "Filtering for smoothness"): pose^(W-1) = reach pose; for j = W-2 .. 0,
 * pose^(j) is the minimum-linear-index chain (joint by joint from the root)
 * among the chains with every joint k in V^(j)_k and within delta + m of
 * joint k of pose^(j+1), for the smallest m >= 0 that admits one.  A
 * waypoint whose survivor set is empty (or whose m would pass max_relax)
 * repeats pose^(j+1) and records m = -1.
 * poses_out [n_way][n_seg + 1][3]; relax_out [n_way][2] = {m, eps2 used};
 * *status = IK_PATH_OK / RELAXED / BROKEN, or UNREACHABLE when the reach
 * pose is not a valid pose of this arm and grid. */
IK_API int ik_plan_path(ik_grid g, const ik_arm* arm, const int32_t* reach_pose, const ik_path_params* pp,
                 int32_t* poses_out, int32_t* relax_out, int* status);

/* The path in the paper's form (sections "Path Planning" and "Filtering for
 * smoothness").  The follower is joint F = n_seg - fold: with fold = 1 the
 * distal end of segment n_seg-1, whose waypoint poses are IK solutions of
 * the arm's first F segments, the last segment being folded along the path;
 * with fold = 0 the end effector.  Its guide points are n_per_seg points per
 * segment of the reach polyline p_0 .. p_F (the i-th point of segment k at
 * p_{k-1} + (i/n)(p_k - p_{k-1}) rounded half up per component, i = 0 ..
 * n-1, then p_F), so n_way = F n_per_seg + 1; the follower lands within
 * squared distance eps2 of its guide point (growing to eps2_max as in
 * ik_plan_path; the last waypoint is p_F itself).  Backward from the reach
 * pose, the pose at waypoint j is the smooth step around pose^(j+1) in which
 * joint k = 1..F moves at most radius[k-1] voxels (-1: joint k is not
 * filtered; the paper filters joints 1 and 2, about half and one waypoint
 * spacing plus slack), all radii growing by one voxel at a time on failure
 * (max_relax as in ik_path_params).  With fold = 1 the last joint of every
 * pose is then the end of an admissible, obstacle-free segment n_seg from the
 * follower, inside the grid, nearest to the point at nominal arc length
 * len[n_seg-1] beyond the guide point along p_0 .. p_n_seg (then the smallest
 * linear index); when none exists the end stays at the follower, the
 * waypoint records -1 and the path is IK_PATH_BROKEN.  reach_pose
 * [n_seg+1][3]; poses_out [n_way][n_seg+1][3]; relax_out [n_way][2] = {radius
 * increments or -1, eps2 used}; *status as for ik_plan_path.  An arm with
 * direction limits (ik_set_segment_limits) is refused with
 * IK_ERR_UNSUPPORTED; unfiltered joints are searched over their whole
 * survivor sets, which is slow on large grids. */
typedef struct {
  int32_t n_per_seg;          /* 1..64 */
  int32_t fold;               /* 0 or 1 */
  int32_t radius[IK_MAX_SEG]; /* radius[k-1] for joint k = 1..F: >= 0, or -1 */
  int32_t eps2, eps2_max, max_relax;
  /* 1: ignore radius[] and take the paper's filter (section "Filtering for
   * smoothness": joint 1 moves about half a waypoint spacing, joint 2 about
   * one, plus one voxel of slack; the other joints unfiltered): with the
   * spacing s = ceil(max_{k <= F} len[k-1] / n_per_seg), radius 1 =
   * ceil(s / 2) + 1, radius 2 = s + 1, the rest -1.  0: radius[] as given. */
  int32_t paper_radii;
} ik_follow_params;
IK_API int ik_plan_path_follow(ik_grid g, const ik_arm* arm, const int32_t* reach_pose,
                               const ik_follow_params* fp, int32_t* poses_out, int32_t* relax_out,
                               int* status);

/* Short reaches (section "Short Reaches"): ik_plan_path with a shorter guide
 * where an early segment meets the target.  For k = 1 .. k_max and, within
 * k, l = 1 .. len[k-1], the virtual arm of the segments len[0] .. len[k-2]
 * and one of length l (its shell from l and arm->tol, so the shell tolerance
 * is the encounter tolerance) is rooted at the root and reaches for the
 * reach pose's end with the reach search of ik_solve_reach; the first one
 * that reaches it (the smallest nominal length) gives the guide polyline
 * (its pose, guide points by the nominal arc rule of its lengths); with none
 * the reach pose is the guide, exactly as in ik_plan_path.  The poses then
 * follow ik_plan_path: pose^(n_way-1) = reach_pose and the smooth steps
 * backward.  shortcut_out [2] = {k, l} ({0, 0}: no shortcut);
 * guide_pose_out nullable [k_max+1][3] (the first k+1 rows are the
 * shortcut's pose when there is one).  k_max in [1, n_seg] (the paper tries
 * segments 1 and 2).  An arm with direction limits is refused with
 * IK_ERR_UNSUPPORTED.  Other arguments and outputs as for ik_plan_path. */
IK_API int ik_plan_path_short(ik_grid g, const ik_arm* arm, const int32_t* reach_pose,
                              const ik_path_params* pp, int k_max, int32_t* poses_out, int32_t* relax_out,
                              int* status, int32_t* shortcut_out, int32_t* guide_pose_out);

/* Path between arbitrary poses (section "Path between Arbitrary Poses"): a
 * virtual arm guide_arm, rooted at the end effector of start_pose, reaches
 * for the target with the reach search of ik_solve_reach; its pose is the
 * polyline the end effector follows (guide points by the nominal-arc rule
 * of guide_arm: g_0 = the start's end effector, g_{n_way-1} = target).
 * pose^(0) = start_pose and poses 1 .. n_way-1 are chained forward, each the
 * smooth step around the previous pose with the relaxation ladder (as in
 * ik_plan_path; T_{n_way-1} = {target}).  start_pose [n_seg+1][3] must lie in
 * the grid (else IK_ERR_ARG); poses_out [n_way][n_seg+1][3]; relax_out
 * [n_way][2]; guide_pose_out nullable [guide n_seg+1][3]; *status =
 * IK_PATH_OK / RELAXED / BROKEN, or UNREACHABLE (every pose the start, m = -1
 * for j >= 1) when the start is not a valid pose of this arm or the virtual
 * arm cannot reach the target. */
IK_API int ik_plan_between(ik_grid g, const ik_arm* arm, const int32_t* start_pose, const ik_arm* guide_arm,
                           const int32_t target[3], const ik_path_params* pp, int32_t* poses_out,
                           int32_t* relax_out, int32_t* guide_pose_out, int* status);

/* Reach + path for n targets sharing one root, all in batched launches with
 * no host round trip between steps: reach survivor sets and poses for all
 * targets, then the survivor sets of all n * n_way waypoints in one batched
 * backward pass per segment, then one smooth-chain block per path.
 * targets [n][3]; reach_out [n][n_seg + 1][3]; found_out [n];
 * poses_out [n][n_way][n_seg + 1][3]; relax_out [n][n_way][2];
 * status_out [n] (IK_PATH_UNREACHABLE when no reach pose exists).  With
 * on_device != 0 every array is a device pointer. */
IK_API int ik_reach_path_many(ik_grid g, const ik_arm* arm, const int32_t root[3], const int32_t* targets,
                       int n, const ik_path_params* pp, int32_t* reach_out, int32_t* found_out,
                       int32_t* poses_out, int32_t* relax_out, int32_t* status_out, int on_device);

/* ------------------------------------------------------ batched graph */
/* A reach + path batch recorded once as a CUDA graph and replayed.  The
 * graph reads n_boxes boxes from boxes_dev and n targets from targets_dev
 * (device, [n][3]) each time it runs, rasterises the occupancy, rebuilds
 * every edge mask and the forward sets, and writes the same outputs as
 * ik_reach_path_many (device arrays, fixed at capture).  A target outside
 * the grid marks an empty slot (found 0, status IK_PATH_UNREACHABLE), so a
 * fixed-size graph serves a varying number of requests.
 * ik_batch_capture runs the batch once normally (sizing every buffer), then
 * records it on the grid's stream, which must not be the legacy default
 * stream (IK_ERR_STATE).  ik_batch_launch enqueues one replay and returns
 * without waiting; the outputs are ready when the grid's stream is.  A
 * replay replaces the grid's occupancy; later ordinary calls on the grid
 * see it. */
typedef struct ik_batch_s* ik_batch;
IK_API int ik_batch_capture(ik_grid g, const ik_arm* arm, const int32_t root[3],
                            const int32_t* boxes_dev, int n_boxes, const int32_t* targets_dev, int n,
                            const ik_path_params* pp, int32_t* reach_dev, int32_t* found_dev,
                            int32_t* poses_dev, int32_t* relax_dev, int32_t* status_dev,
                            ik_batch* out);
IK_API int ik_batch_launch(ik_batch b);
IK_API int ik_batch_destroy(ik_batch b);

/* ------------------------------------------------------- uneven batch */
/* One independent reach + path problem of an uneven batch: its own grid
 * (extents as in ik_create_grid), boxes (host, [n_boxes][6], inclusive),
 * arm, root, target and waypoint count. */
typedef struct {
  int32_t nx, ny, nz;
  const int32_t* boxes;
  int32_t n_boxes;
  int32_t n_seg;
  const int32_t* len;
  float tol;
  int32_t root[3];
  int32_t target[3];
  int32_t n_way;
} ik_problem;

/* Path rules shared by the batch (as in ik_path_params); blocks_per_sm: the
 * persistent kernel's resident blocks per SM (0 or 1: one). */
typedef struct {
  int32_t delta, eps2, eps2_max, max_relax;
  int32_t blocks_per_sm;
} ik_batch_params;

/* Sizes (int32 counts) of the packed outputs of ik_solve_batch. */
IK_API int ik_batch_output_sizes(const ik_problem* probs, int n, size_t* reach_ints,
                                 size_t* poses_ints, size_t* relax_ints);

/* An engine for uneven batches on the current device: it keeps the shell
 * tables, the device pool, the work queue and the pinned staging between
 * calls (allocated when a call first needs them, reused afterwards).  Not
 * thread-safe across concurrent calls on one engine beyond an internal lock.
 * Destroying an engine waits for the device. */
typedef struct ik_batch_engine_s* ik_batch_engine;
IK_API int ik_batch_engine_create(ik_batch_engine* out);
IK_API int ik_batch_engine_destroy(ik_batch_engine e);
/* Pool bytes one launch may use (0: 70 % of the device's free memory at the
 * first call); a batch that needs more runs as several launches in problem
 * order. */
IK_API int ik_batch_engine_set_budget(ik_batch_engine e, size_t pool_bytes);
/* How long (ns, at least 1000; default 20 s) a launch waits with no work
 * item completing anywhere before it gives up: its blocks then stop taking
 * items and the unfinished problems report IK_ERR_TIMEOUT in job_rc. */
IK_API int ik_batch_engine_set_timeout(ik_batch_engine e, int64_t ns);
/* on = 1 (default): on the waypoint levels whose tiles leave room for a
 * third halo in shared memory, a work item carries two waypoint queries of
 * a problem, which share each segment test's supercover walk; 0: one query
 * per item.  Results are identical. */
IK_API int ik_batch_engine_set_pairs(ik_batch_engine e, int on);

/* Solve n uneven problems (the systems pattern of batching, no paper
 * counterpart; every problem follows exactly the rules of ik_solve_reach +
 * ik_plan_path on its own grid, sections "The procedure for IK solution",
 * "Smooth sequence computation" and "Filtering for smoothness"; segment
 * tests walk the supercover, no edge masks are stored).  Asynchronous on
 * cuda_stream (NULL: the legacy default stream): the call copies the host
 * inputs (probs and their boxes and lengths) to pinned staging and device
 * memory in stream order, clears the engine's pool, and launches ONE
 * persistent kernel whose resident blocks take work items (rasterise slabs,
 * seeds, propagation tiles of every level of every problem, tracebacks,
 * guide points, smooth chains) from a device queue; the block that finishes
 * a stage of a problem queues that problem's next stage.  Outputs are device
 * pointers, packed in problem order: found [n], status [n] (an IK_PATH_*
 * code), reach [(n_seg+1)*3 per problem], poses [n_way*(n_seg+1)*3 per
 * problem], relax [n_way*2 per problem] (sizes from ik_batch_output_sizes),
 * and job_rc [n]: IK_OK when the problem finished, IK_ERR_TIMEOUT when the
 * launch gave up (ik_batch_engine_set_timeout).  Every segment length must
 * keep the shell's reach within 31 voxels (else IK_ERR_UNSUPPORTED), and at
 * most 8192 boxes per problem.  Returns IK_ERR_ARG / IK_ERR_OOM /
 * IK_ERR_CUDA when enqueueing fails. */
IK_API int ik_solve_batch_async(ik_batch_engine e, const ik_problem* probs, int n, const ik_batch_params* bp,
                                int32_t* found_dev, int32_t* reach_dev, int32_t* poses_dev,
                                int32_t* relax_dev, int32_t* status_dev, int32_t* job_rc_dev,
                                void* cuda_stream);

/* The same, synchronous, with host outputs, on a per-device engine that the
 * library keeps for the process (its memory grows to the largest batch and
 * is reused).  gpu_ms_out (nullable) receives the device time from the
 * first upload to the end of the last launch.  Returns the first job's
 * error (IK_ERR_TIMEOUT) if any problem did not finish. */
IK_API int ik_solve_batch(const ik_problem* probs, int n, const ik_batch_params* bp,
                          int32_t* found_out, int32_t* reach_out, int32_t* poses_out,
                          int32_t* relax_out, int32_t* status_out, double* gpu_ms_out);

/* The uneven batch as a CUDA graph: ik_batch_capture_uneven plans the n
 * problems (as ik_solve_batch_async), copies their descriptors, boxes and
 * initial work queue into device memory the graph owns (synchronously,
 * before returning), and captures -- on a stream of its own -- the
 * sequence that resets the queue, clears the problems' working memory,
 * fills job_rc_dev with IK_ERR_TIMEOUT and runs the persistent kernel: one
 * launch.  ik_batch_graph_launch replays it on cuda_stream (NULL: the
 * legacy default stream) and returns without waiting; every replay writes
 * the same outputs to the same device arrays (the layout of
 * ik_batch_output_sizes), which must stay allocated while the graph
 * exists.  The problems' data are copied at capture: the caller's arrays
 * may change afterwards.  The whole batch must fit one launch (the
 * engine's pool budget), else IK_ERR_UNSUPPORTED.  The graph takes the
 * engine's timeout and query-pair setting at capture.  Returns IK_OK,
 * IK_ERR_ARG, IK_ERR_UNSUPPORTED, IK_ERR_OOM or IK_ERR_CUDA; a graph
 * handle is freed by ik_batch_graph_destroy (which waits for the device). */
typedef struct ik_batch_graph_s* ik_batch_graph;
IK_API int ik_batch_capture_uneven(ik_batch_engine e, const ik_problem* probs, int n, const ik_batch_params* bp,
                                   int32_t* found_dev, int32_t* reach_dev, int32_t* poses_dev,
                                   int32_t* relax_dev, int32_t* status_dev, int32_t* job_rc_dev,
                                   ik_batch_graph* out);
IK_API int ik_batch_graph_launch(ik_batch_graph g, void* cuda_stream);
IK_API int ik_batch_graph_destroy(ik_batch_graph g);

/* ------------------------------------------------------------- replan */
/* Validity of n poses under the current occupancy: every joint inside the
 * grid, every offset in its shell, every segment obstacle-free.
 * poses [n][n_seg + 1][3]; valid_out [n] (1 / 0). */
IK_API int ik_validate_poses(ik_grid g, const ik_arm* arm, const int32_t* poses, int n, int32_t* valid_out);

/* Midcourse replan under the current occupancy (section "Dynamic
 * Obstacles").  The arm is at waypoint current_idx of poses_in
 * [n_way][n_seg + 1][3].  If every later pose is still valid the path is
 * kept (IK_PATH_KEPT).  Otherwise poses 0..current_idx are kept; the reach
 * pose is kept if valid, else re-solved joint by joint from the root taking
 * the successor in V_k closest to the old joint (squared distance, then
 * linear index), the path's least-distance objective; guide points come
 * from that reach pose; and poses current_idx+1 .. n_way-1 are chained
 * forward from pose^(current_idx) by the smooth-step rule of ik_plan_path.
 * IK_PATH_UNREACHABLE (poses after current_idx repeat it, m = -1) when the
 * target cannot be reached now. */
IK_API int ik_replan(ik_grid g, const ik_arm* arm, const int32_t* poses_in, int n_way, int current_idx,
              const ik_path_params* pp, int32_t* poses_out, int32_t* relax_out, int* status);

/* ------------------------------------------------ allocation-free variant */
/* Forward reachable sets F_0..F_S, like ik_forward_sets, for callers that
 * cannot allocate GPU memory when they need the answer (a caching or arena
 * allocator owns the device, a real-time loop must not pay cudaMalloc's
 * synchronisation, or allocation is forbidden after start-up).  The paper
 * has no counterpart: this is a deployment interface only.
 *
 * occ_words (device, bit-packed occupancy, 1 = occupied) and fsets_out
 * (device, [n_seg + 1][(nx/32) * ny * nz] words) belong to the caller; arm
 * and root are host memory.  The grid rules are those of ik_create_grid.
 * The call allocates nothing: its scratch -- the arm's shell offsets and
 * supercover lists -- is one fixed array of 4.25 MiB in the library's device
 * memory (held by every GPU that loads the library until the process ends).
 * Limits: at most 32768 shell offsets over all segments and 2^20 supercover
 * voxels (the arms {8,7,6,5} and {20,18,16,14,12,10,8,6} fit, six segments
 * of length 20 fit); larger arms return IK_ERR_UNSUPPORTED.  Segment tests walk the supercover
 * against the occupancy instead of reading stored edge masks.
 *
 * The first call on a device looks up the array's device address (with
 * that device current) and should come before any stream capture.  Every
 * call shares the array and overwrites the part it uses; calls whose work
 * overlaps on the GPU (other streams, other threads) race on it.  Host
 * threads are serialised by a lock while the tables are built and copied,
 * but the kernels of two calls still race if their streams overlap.  The
 * call is synchronous on cuda_stream (NULL: the legacy default stream).
 * Returns IK_OK, IK_ERR_ARG, IK_ERR_UNSUPPORTED, IK_ERR_OOM (a CUDA call
 * reported cudaErrorMemoryAllocation) or IK_ERR_CUDA. */
IK_API int ik_forward_sets_noalloc(const uint32_t* occ_words, int nx, int ny, int nz,
                                   const ik_arm* arm, const int32_t root[3], uint32_t* fsets_out,
                                   void* cuda_stream);

/* ------------------------------------------------------------- profiling */
/* Per-kernel-class timing: with timing != 0 every launch is bracketed by two
 * CUDA events recorded on the grid's stream; with counting != 0 the
 * propagation kernels also count their work (slower; for measurement runs
 * only).  Off by default. */
IK_API int ik_profile_enable(ik_grid g, int timing, int counting);
/* Totals since the last read, per kernel class i < cap: ms_out[i] summed
 * event time, launches_out[i] number of launches, counters_out[8*i + 0..7]
 * = (offset-word pairs visited, pairs with a non-zero shifted input word,
 * edge-mask words read, output words with a non-empty mask, warp-level
 * offset iterations, blocks that did work, warps of the tiled kernels that
 * walked the offsets, the lanes of those warps with a non-empty mask); any
 * output may be NULL.
 * Returns the number of kernel classes, or a negative error. */
IK_API int ik_profile_read(ik_grid g, double* ms_out, int64_t* launches_out, uint64_t* counters_out,
                           int cap);
/* Name of kernel class i ("" when out of range). */
IK_API const char* ik_profile_name(int i);

/* Replans of n live paths at once, with every decision taken on the GPU
 * (the rules of ik_replan, applied per slot): poses_in [n][n_way][n_seg+1][3]
 * (every pose starting at root), current [n] (the arm's waypoint per slot;
 * a value outside [0, n_way) marks an empty slot, whose status is -1).
 * Outputs poses_out [n][n_way][n_seg+1][3], relax_out [n][n_way][2],
 * status_out [n].  With on_device != 0 every array is a device pointer (and
 * the root is not checked against the poses). */
IK_API int ik_replan_many(ik_grid g, const ik_arm* arm, const int32_t root[3], const int32_t* poses_in,
                          const int32_t* current, int n, const ik_path_params* pp,
                          int32_t* poses_out, int32_t* relax_out, int32_t* status_out, int on_device);

/* ------------------------------------------------------- peak probes */
/* Measured peaks for the rooflines of the boolean propagation (the paper
 * gives no hardware figures for its GPU; section "Implementation
 * Performance" only reports times).  Runs one throughput probe on the
 * current device, enqueued on cuda_stream (NULL: legacy default stream) and
 * waited for: kind 0 = 3-input logic ops (lop3.b32), kind 1 = funnel shifts
 * (shf.r.wrap.b32), kind 2 = conflict-free 32-bit shared-memory word loads.
 * blocks_per_sm (1..8) blocks of 256 threads per SM run iters (1..2^24)
 * iterations of 128 (kinds 0, 1) or 32 (kind 2) ops per thread.  Outputs
 * (nullable): ops_per_s_out = counted ops / event time; ms_out = event time;
 * sm_mhz_out = the SM clock the first block saw (clock64 ticks per
 * %globaltimer microsecond).  Allocates a few bytes of device memory per
 * call.  Returns IK_OK, IK_ERR_ARG or IK_ERR_CUDA. */
IK_API int ik_probe_peak(int kind, int blocks_per_sm, int iters, void* cuda_stream, double* ops_per_s_out,
                         double* ms_out, double* sm_mhz_out);

/* ------------------------------------------------------- host utilities */
/* Shell bounds and offsets of one segment length, as the library builds
 * them (offsets ordered by |d|^2, then z, y, x).  Writes up to cap offsets
 * (x, y, z) and returns the shell size, or a negative error code. */
IK_API int ik_shell_offsets(int len, float tol, int32_t* lo2_hi2, int32_t* offs_out, int cap);
/* Closed supercover of the segment 0 -> d as the library builds it (by an
 * incremental integer traversal of the segment's boundary crossings),
 * ordered by (z, y, x).  Returns its size or a negative error code. */
IK_API int ik_supercover_offsets(const int32_t d[3], int32_t* vox_out, int cap);
/* The row-lane propagation's offset table of the shell of one segment
 * length (IK_OPT_ROW_LANES), as the library builds it on the host: *R_out =
 * the shell's reach; offs_out [n][3] = the offsets in device order (the
 * order of the edge-mask rows: by (z, y, x)); tabr_out [n] = the entries,
 * per dz plane the offsets with dx < 0 then those with dx >= 0, each run
 * ordered by (dy, dx), entry (e << 11) | ((dy + 32) << 5) | (dx & 31), e
 * the offset's device index; rowsr_out [(2R+1) * 2 * (2R+2)] = the start of
 * each (dz, sign, dy) run, entry 2R+1 of a (dz, sign) run its end.  At most
 * cap offsets and rowsr_cap starts are written (nullable outputs).  Returns
 * n, IK_ERR_ARG, or IK_ERR_UNSUPPORTED when the reach exceeds 31 (no
 * table). */
IK_API int ik_row_table(int len, float tol, int32_t* R_out, int32_t* offs_out, int32_t* tabr_out, int cap,
                        int32_t* rowsr_out, int rowsr_cap);
/* The row-lane edge masks' supercover table of the same shell (section
 * "Testing for collisions": the voxels a segment crosses), as the library
 * builds it: sc_start_out [n + 1] = where each offset's voxels start (device
 * order, as ik_row_table's offsets); sctabr_out [m] = per voxel v,
 * ((v.z * (32 + 2R) + v.y) << 6) | (v.x + 32).  At most cap_off starts and
 * cap_sc voxels are written (nullable outputs).  Returns m, IK_ERR_ARG, or
 * IK_ERR_UNSUPPORTED when the reach exceeds 31. */
IK_API int ik_row_mask_table(int len, float tol, int32_t* sc_start_out, int cap_off, int32_t* sctabr_out,
                             int cap_sc);

#ifdef __cplusplus
}
#endif

#endif /* IK_B300_H */
