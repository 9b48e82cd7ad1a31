// C ABI of the library: argument checks, device-resident state per grid, and
// the launch sequences of the hot path.  No step of the method runs on the
// host: the host builds the integer shell/supercover tables once per segment
// length and then only enqueues kernels and copies.

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <map>
#include <string>
#include <vector>

#include "ik_internal.h"

using namespace ikb;

namespace {

thread_local std::string g_last_error;

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

struct GridState;

}  // namespace

namespace ikb {
// The row-lane propagation's table of shell h (tabr, rowsr of SegDev),
// empty when the reach exceeds 31: per dz plane the offsets with dx < 0,
// then those with dx >= 0, each run ordered by (dy, dx) (the device order
// within a (dz, dy) row is by dx), with the run starts per dy.
void build_row_table(const ShellHost& h, std::vector<int32_t>* tabr, std::vector<int32_t>* rowsr) {
  tabr->clear();
  rowsr->clear();
  const int R = h.R;
  if (R > 31) return;
  const int side = 2 * R + 1, rs = 2 * R + 2;
  tabr->reserve(h.dev_off.size());
  rowsr->assign((size_t)side * 2 * rs, 0);
  for (int dz = -R; dz <= R; ++dz)
    for (int neg = 1; neg >= 0; --neg) {
      int32_t* run = rowsr->data() + ((size_t)(dz + R) * 2 + (1 - neg)) * rs;
      for (int dy = -R; dy <= R; ++dy) {
        run[dy + R] = (int32_t)tabr->size();
        const int r = (dz + R) * side + (dy + R);
        for (int i = h.rows[r]; i < h.rows[r + 1]; ++i) {
          const int dx = unpack_x(h.dev_off[i]);
          if ((dx < 0) != (neg == 1)) continue;
          tabr->push_back((int32_t)(((uint32_t)i << 11) | ((uint32_t)(dy + 32) << 5) | (uint32_t)(dx & 31)));
        }
      }
      run[2 * R + 1] = (int32_t)tabr->size();
    }
}
// The row-lane edge masks' supercover table of shell h (empty when the
// reach exceeds 31): per supercover voxel (v of h.sc, in its order),
// ((vz * (32 + 2R) + vy) << 6) | (vx + 32).
void build_row_mask_table(const ShellHost& h, std::vector<int32_t>* sctabr) {
  sctabr->clear();
  if (h.R > 31) return;
  const int RY = 32 + 2 * h.R;
  sctabr->resize(h.sc.size());
  for (size_t i = 0; i < h.sc.size(); ++i) {
    const int32_t v = h.sc[i];
    const int vx = unpack_x(v), vy = unpack_y(v), vz = unpack_z(v);
    (*sctabr)[i] = (int32_t)(((uint32_t)(vz * RY + vy) << 6) | (uint32_t)(vx + 32));
  }
}
void note_cuda_error(cudaError_t e) { g_last_error = cudaGetErrorString(e); }
}  // namespace ikb

struct ik_grid_s {
  int device = 0;
  Dims d{};
  TileCfg tc{};
  cudaStream_t st = nullptr;
  uint32_t* d_occ = nullptr;      // the occupancy every kernel reads (dilated when asked)
  uint32_t* d_occ_raw = nullptr;  // the occupancy as set, before dilation
  int dilate_r2 = 0;
  int work_list = 1;              // IK_OPT_WORK_LIST
  int use_tma = 0;                // IK_OPT_TMA_MASKS (off: measured slower, see the header)
  std::map<int, CUtensorMap> tmaps;  // TMA tensor maps over d_occ, per shell reach
  int* d_tma_slow = nullptr;      // blocks whose TMA copy did not complete in time
  uint64_t version = 1;
  std::map<std::pair<int, int>, ShellDev*> shells;
  // shells restricted to an approach cone: (lo2, hi2, ax, ay, az, num, den)
  std::map<std::array<int, 7>, ShellDev*> cone_shells;
  // per-segment direction limits, by arm (n_seg, lengths, tol bits)
  std::map<std::vector<int32_t>, std::vector<ik_cone>> limits;
  // forward-set cache
  bool f_valid = false;
  int f_root[3] = {0, 0, 0};
  std::vector<std::pair<int, int>> f_key;
  uint64_t f_version = 0;
  DevBuf F;
  // scratch
  DevBuf V, Vw, chain, boxes;
  DevBuf F_box, V_box, Vw_box;  // word boxes of every set (min form)
  DevBuf b_root, b_targets, b_reach, b_found, b_poses, b_relax, b_status, b_eps, b_g, b_valid;
  DevBuf b_old;
  DevBuf b_rp, b_rin, b_rc;  // batched replan: bookkeeping, host-form inputs
  DevBuf b_list;             // work list of the batched propagations
  DevBuf b_tposes, b_fold;   // follower path: poses of the follower's joints, fold points
  int num_sms = 148;
  // per-kernel profiling: events recorded on st around each launch
  bool prof_on = false, count_on = false;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  struct Rec {
    int id;
    cudaEvent_t a, b;
  };
  std::vector<Rec> recs;
  unsigned long long* d_counters = nullptr;
  std::vector<unsigned long long> h_counters;  // counts known on the host at launch time
  bool capturing = false;  // inside ik_batch_capture: no allocation, no host transfer
  bool use_masks = true;   // store per-offset edge masks (else walk supercovers on the fly)
  // Captured batches hold device pointers of this grid.  A buffer replaced
  // while any batch lives is retired (freed when the last batch goes), and
  // every replacement or mask-layout change bumps buf_gen, so that a replay
  // knows whether its buffers are still the grid's.
  int live_batches = 0;
  std::vector<void*> retired;
  uint64_t buf_gen = 0;
};

struct ik_batch_s {
  ik_grid g = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int root[3] = {0, 0, 0};
  std::vector<std::pair<int, int>> key;  // the arm's shells
  std::vector<ShellDev*> used;           // every table whose masks the graph rebuilds
  uint64_t gen = 0;                      // the grid's buf_gen at capture
  int32_t* d_root = nullptr;             // device copy of root, read by the graph
};

namespace {

#define CK(call)                                      \
  do {                                                \
    cudaError_t _e = (call);                          \
    if (_e != cudaSuccess) return fail_cuda(_e);      \
  } while (0)

int fail_cuda(cudaError_t e) {
  g_last_error = cudaGetErrorString(e);
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();  // clear the sticky-free allocation error
    return IK_ERR_OOM;
  }
  return IK_ERR_CUDA;
}

// The occupancy, edge masks and forward sets were rewritten by a replayed
// graph: forget what the host knew about them.
void forget_device_state(ik_grid g) {
  ++g->version;
  g->f_valid = false;
  for (auto& kv : g->shells) kv.second->mask_version = ~0ull;
  for (auto& kv : g->cone_shells) kv.second->mask_version = ~0ull;
}

enum ProfId {
  P_RASTER,
  P_MASKS,
  P_FWD,
  P_BWD_REACH,
  P_BWD_WAY,
  P_SEED,
  P_TRACE,
  P_GUIDE,
  P_CHAIN,
  P_VALIDATE,
  P_TILE_LIST,
  P_WAY_K1,  // waypoint backward pass per segment level k = 1 .. IK_MAX_SEG
  P_N = P_WAY_K1 + IK_MAX_SEG
};
const char* kProfNames[P_N] = {"rasterize",
                               "edge_masks",
                               "propagate_forward",
                               "propagate_backward_reach",
                               "propagate_backward_waypoints",
                               "seed",
                               "traceback",
                               "guide_targets",
                               "smooth_chain",
                               "validate",
                               "tile_list",
                               "way_k1", "way_k2", "way_k3", "way_k4", "way_k5", "way_k6",
                               "way_k7", "way_k8", "way_k9", "way_k10", "way_k11", "way_k12",
                               "way_k13", "way_k14", "way_k15", "way_k16"};

cudaEvent_t take_event(ik_grid g) {
  if (g->ev_used == g->ev_pool.size()) {
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    g->ev_pool.push_back(e);
  }
  return g->ev_pool[g->ev_used++];
}

// Records an event before and after the launches in its scope when
// profiling is on; the pair is resolved by ik_profile_read.
struct ProfScope {
  ik_grid g;
  int id;
  cudaEvent_t a = nullptr;
  ProfScope(ik_grid g_, int id_) : g(g_), id(id_) {
    if (id >= 0 && g->prof_on && (a = take_event(g))) cudaEventRecord(a, g->st);
  }
  ~ProfScope() {
    if (!a) return;
    cudaEvent_t b = take_event(g);
    if (!b) return;
    cudaEventRecord(b, g->st);
    g->recs.push_back({id, a, b});
  }
};

constexpr int kCounters = 8;

unsigned long long* counters(ik_grid g, int id) {
  return (g->count_on && g->d_counters) ? g->d_counters + kCounters * id : nullptr;
}

// Grow a device buffer to at least `bytes`; contents are not kept.  With
// `zero`, a newly allocated buffer is cleared.
// Gives up a device buffer: freed, or kept for the captured batches that
// still write it.
int release(ik_grid g, void* p) {
  if (!p) return IK_OK;
  ++g->buf_gen;
  if (g->live_batches > 0) {
    g->retired.push_back(p);
    return IK_OK;
  }
  CK(cudaStreamSynchronize(g->st));
  CK(cudaFree(p));
  return IK_OK;
}

int ensure(ik_grid g, DevBuf& b, size_t bytes, bool zero = false) {
  if (bytes == 0) bytes = 16;
  if (b.bytes >= bytes) return IK_OK;
  if (g->capturing) return IK_ERR_STATE;  // buffers are sized by the warm-up run
  if (b.p) {
    int rc = release(g, b.p);
    if (rc) return rc;
    b.p = nullptr;
    b.bytes = 0;
  }
  cudaError_t e = cudaMalloc(&b.p, bytes);
  if (e != cudaSuccess) {
    b.p = nullptr;
    return fail_cuda(e);
  }
  b.bytes = bytes;
  if (zero) CK(cudaMemsetAsync(b.p, 0, bytes, g->st));
  return IK_OK;
}

template <typename T>
T* ptr(DevBuf& b) {
  return reinterpret_cast<T*>(b.p);
}

int to_device(ik_grid g, DevBuf& b, const void* src, size_t bytes) {
  int rc = ensure(g, b, bytes);
  if (rc) return rc;
  CK(cudaMemcpyAsync(b.p, src, bytes, cudaMemcpyHostToDevice, g->st));
  return IK_OK;
}

int check_arm(const ik_arm* arm) {
  if (!arm || !arm->len || arm->n_seg < 1 || arm->n_seg > IK_MAX_SEG) return IK_ERR_ARG;
  if (!(arm->tol >= 0.0f && arm->tol < 1.0f)) return IK_ERR_ARG;
  for (int k = 0; k < arm->n_seg; ++k)
    if (arm->len[k] < 1 || arm->len[k] > IK_MAX_LEN) return IK_ERR_ARG;
  return IK_OK;
}

// Shell table for (lo2, hi2) (restricted to `cone` when given), built on the
// host and uploaded.
int make_shell(ik_grid g, int lo2, int hi2, const ConeSpec* cone, ShellDev** out) {
  ShellDev* s = new ShellDev();
  build_shell(lo2, hi2, &s->host, cone);
  const size_t n = s->host.off.size();
  if (n == 0) {
    delete s;
    return IK_ERR_ARG;
  }
  s->reach = s->host.R;
  // shared-memory deltas of the tiled propagation for this grid's pitch
  std::vector<int32_t> tab(n);
  for (size_t i = 0; i < n; ++i) {
    const int32_t o = s->host.dev_off[i];
    const int dx = unpack_x(o), dy = unpack_y(o);
    const int delta = dy * g->tc.P + (dx >> 5);
    tab[i] = (int32_t)(((uint32_t)delta << 5) | (uint32_t)(dx & 31));
  }
  // shared-memory deltas of every supercover voxel for the tiled edge masks
  const int RY = g->tc.TY + 2 * s->reach;
  std::vector<int32_t> sctab(s->host.sc.size());
  for (size_t i = 0; i < sctab.size(); ++i) {
    const int32_t v = s->host.sc[i];
    const int vx = unpack_x(v), vy = unpack_y(v), vz = unpack_z(v);
    const int delta = (vz * RY + vy) * g->tc.P + (vx >> 5);
    sctab[i] = (int32_t)((uint32_t)delta << 5) | (vx & 31);
  }
  // and for rows staged without pad words (pitch wx), when a warp covers
  // whole rows: the word offset, the sign of dx and the shift
  std::vector<int32_t> tabw;
  const int wxw = g->d.wx;
  if (32 % wxw == 0) {
    tabw.resize(n);
    for (size_t i = 0; i < n; ++i) {
      const int32_t o = s->host.dev_off[i];
      const int dx = unpack_x(o), dy = unpack_y(o);
      const int delta = dy * wxw + (dx >> 5);
      tabw[i] = (int32_t)(((uint32_t)delta << 6) | ((uint32_t)(dx < 0) << 5) | (uint32_t)(dx & 31));
    }
  }
  // and for the row-lane propagation (reach at most 31)
  std::vector<int32_t> tabr, rowsr;
  build_row_table(s->host, &tabr, &rowsr);
  // and for the row-lane edge masks (rows of 32 + 2R per halo slice)
  std::vector<int32_t> sctabr;
  build_row_mask_table(s->host, &sctabr);
  // and for the TMA-staged brick (pitch BX, word w at column w + 4)
  const int BX = tma_mask_pitch(g->d);
  std::vector<int32_t> sctab_tma;
  if (BX > 0) {
    sctab_tma.resize(s->host.sc.size());
    for (size_t i = 0; i < sctab_tma.size(); ++i) {
      const int32_t v = s->host.sc[i];
      const int vx = unpack_x(v), vy = unpack_y(v), vz = unpack_z(v);
      const int delta = (vz * RY + vy) * BX + (vx >> 5);
      sctab_tma[i] = (int32_t)((uint32_t)delta << 5) | (vx & 31);
    }
  }
  cudaError_t e = cudaMalloc(&s->d_off, n * 4);
  if (e == cudaSuccess) e = cudaMalloc(&s->d_tab, n * 4);
  if (e == cudaSuccess) e = cudaMalloc(&s->d_sctab, sctab.size() * 4);
  if (e == cudaSuccess && BX > 0) e = cudaMalloc(&s->d_sctab_tma, sctab_tma.size() * 4);
  if (e == cudaSuccess && !tabw.empty()) e = cudaMalloc(&s->d_tabw, n * 4);
  if (e == cudaSuccess && !tabr.empty()) e = cudaMalloc(&s->d_tabr, n * 4);
  if (e == cudaSuccess && !tabr.empty()) e = cudaMalloc(&s->d_rowsr, rowsr.size() * 4);
  if (e == cudaSuccess && !sctabr.empty()) e = cudaMalloc(&s->d_sctabr, sctabr.size() * 4);
  if (e == cudaSuccess) e = cudaMalloc(&s->d_rows, s->host.rows.size() * 4);
  if (e == cudaSuccess) e = cudaMalloc(&s->d_sc_start, (n + 1) * 4);
  if (e == cudaSuccess) e = cudaMalloc(&s->d_sc, s->host.sc.size() * 4);
  if (e != cudaSuccess) {
    cudaFree(s->d_off);
    cudaFree(s->d_tab);
    cudaFree(s->d_sctab);
    cudaFree(s->d_sctab_tma);
    cudaFree(s->d_tabw);
    cudaFree(s->d_tabr);
    cudaFree(s->d_rowsr);
    cudaFree(s->d_sctabr);
    cudaFree(s->d_rows);
    cudaFree(s->d_sc_start);
    cudaFree(s->d_sc);
    delete s;
    return fail_cuda(e);
  }
  CK(cudaMemcpyAsync(s->d_tab, tab.data(), n * 4, cudaMemcpyHostToDevice, g->st));
  CK(cudaMemcpyAsync(s->d_sctab, sctab.data(), sctab.size() * 4, cudaMemcpyHostToDevice, g->st));
  if (BX > 0)
    CK(cudaMemcpyAsync(s->d_sctab_tma, sctab_tma.data(), sctab_tma.size() * 4, cudaMemcpyHostToDevice, g->st));
  if (!tabw.empty())
    CK(cudaMemcpyAsync(s->d_tabw, tabw.data(), n * 4, cudaMemcpyHostToDevice, g->st));
  if (!sctabr.empty())
    CK(cudaMemcpyAsync(s->d_sctabr, sctabr.data(), sctabr.size() * 4, cudaMemcpyHostToDevice, g->st));
  if (!tabr.empty()) {
    CK(cudaMemcpyAsync(s->d_tabr, tabr.data(), n * 4, cudaMemcpyHostToDevice, g->st));
    CK(cudaMemcpyAsync(s->d_rowsr, rowsr.data(), rowsr.size() * 4, cudaMemcpyHostToDevice, g->st));
  }
  CK(cudaMemcpyAsync(s->d_off, s->host.dev_off.data(), n * 4, cudaMemcpyHostToDevice, g->st));
  CK(cudaMemcpyAsync(s->d_rows, s->host.rows.data(), s->host.rows.size() * 4, cudaMemcpyHostToDevice,
                     g->st));
  CK(cudaMemcpyAsync(s->d_sc_start, s->host.sc_start.data(), (n + 1) * 4, cudaMemcpyHostToDevice, g->st));
  CK(cudaMemcpyAsync(s->d_sc, s->host.sc.data(), s->host.sc.size() * 4, cudaMemcpyHostToDevice, g->st));
  CK(cudaStreamSynchronize(g->st));
  *out = s;
  return IK_OK;
}

int get_shell(ik_grid g, int lo2, int hi2, ShellDev** out) {
  auto key = std::make_pair(lo2, hi2);
  auto it = g->shells.find(key);
  if (it != g->shells.end()) {
    *out = it->second;
    return IK_OK;
  }
  int rc = make_shell(g, lo2, hi2, nullptr, out);
  if (rc) return rc;
  g->shells[key] = *out;
  return IK_OK;
}

int get_cone_shell(ik_grid g, int lo2, int hi2, const ik_cone& c, ShellDev** out) {
  const std::array<int, 7> key{lo2, hi2, c.axis[0], c.axis[1], c.axis[2], c.cos2_num, c.cos2_den};
  auto it = g->cone_shells.find(key);
  if (it != g->cone_shells.end()) {
    *out = it->second;
    return IK_OK;
  }
  const ConeSpec cs{c.axis[0], c.axis[1], c.axis[2], c.cos2_num, c.cos2_den};
  int rc = make_shell(g, lo2, hi2, &cs, out);
  if (rc) return rc;
  g->cone_shells[key] = *out;
  return IK_OK;
}

int check_cone(const ik_cone* c) {
  if (!c) return IK_OK;
  const int* a = c->axis;
  if (a[0] == 0 && a[1] == 0 && a[2] == 0) return IK_ERR_ARG;
  for (int i = 0; i < 3; ++i)
    if (a[i] < -1024 || a[i] > 1024) return IK_ERR_ARG;
  if (c->cos2_den < 1 || c->cos2_den > 1000000 || c->cos2_num < 0 || c->cos2_num > c->cos2_den)
    return IK_ERR_ARG;
  return IK_OK;
}

// Edge masks of a shell for the current occupancy over (at least) the word
// box `need`; recomputed when stale.  Masks still valid for another box keep
// it: the new box is the union of both.
// cuTensorMapEncodeTiled, reached through the runtime (no link to the driver
// library); nullptr when the driver does not offer it.
PFN_cuTensorMapEncodeTiled_v12000 tma_encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      p = nullptr;
    }
    return (PFN_cuTensorMapEncodeTiled_v12000)p;
  }();
  return fn;
}

// The tensor map over the grid's occupancy for bricks of shell reach R
// (nullptr when the TMA form does not apply).
const CUtensorMap* occ_tmap(ik_grid g, int R) {
  auto it = g->tmaps.find(R);
  if (it != g->tmaps.end()) return &it->second;
  const int BX = tma_mask_pitch(g->d);
  PFN_cuTensorMapEncodeTiled_v12000 fn = tma_encode_fn();
  if (BX <= 0 || !fn) return nullptr;
  const Dims& d = g->d;
  CUtensorMap m;
  cuuint64_t dims[3] = {(cuuint64_t)d.wx, (cuuint64_t)d.ny, (cuuint64_t)d.nz};
  cuuint64_t strides[2] = {(cuuint64_t)d.wx * 4, (cuuint64_t)d.wx * d.ny * 4};
  cuuint32_t box[3] = {(cuuint32_t)BX, (cuuint32_t)(g->tc.TY + 2 * R), (cuuint32_t)(g->tc.TZ + 2 * R)};
  cuuint32_t es[3] = {1, 1, 1};
  if (fn(&m, CU_TENSOR_MAP_DATA_TYPE_UINT32, 3, (void*)g->d_occ, dims, strides, box, es,
         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return nullptr;
  return &g->tmaps.emplace(R, m).first->second;
}

// Edge masks of shell s over box b: the TMA-staged form where it applies
// (and IK_OPT_TMA_MASKS is on), else the per-thread staging.
cudaError_t launch_masks(ik_grid g, const ShellDev& s, const MaskBox& b, uint32_t* mask) {
  if (g->use_tma && s.d_sctab_tma && tma_mask_smem_bytes(g->tc, s.reach, tma_mask_pitch(g->d)) > 0) {
    const CUtensorMap* m = occ_tmap(g, s.reach);
    if (m) return launch_edge_masks_tma(g->d, g->tc, m, g->d_occ, s, b, mask, g->d_tma_slow, g->st);
  }
  return launch_edge_masks(g->d, g->tc, g->d_occ, s, b, mask, g->st);
}

int ensure_masks(ik_grid g, ShellDev* s, const MaskBox& need) {
  const bool valid = s->d_mask && s->mask_version == g->version;
  if (valid && s->mbox.contains(need)) return IK_OK;
  if (g->capturing) return IK_ERR_STATE;
  MaskBox b = need;
  if (valid) {
    b.wx0 = std::min(b.wx0, s->mbox.wx0);
    b.y0 = std::min(b.y0, s->mbox.y0);
    b.z0 = std::min(b.z0, s->mbox.z0);
    b.wx1 = std::max(b.wx1, s->mbox.wx1);
    b.y1 = std::max(b.y1, s->mbox.y1);
    b.z1 = std::max(b.z1, s->mbox.z1);
  }
  const size_t bytes = s->host.off.size() * (size_t)b.words() * 4;
  if (bytes > s->mask_bytes) {
    int rc = release(g, s->d_mask);
    if (rc) return rc;
    s->d_mask = nullptr;
    s->mask_bytes = 0;
    cudaError_t e = cudaMalloc(&s->d_mask, bytes);
    if (e != cudaSuccess) {
      s->d_mask = nullptr;
      return fail_cuda(e);
    }
    s->mask_bytes = bytes;
  }
  if (memcmp(&b, &s->mbox, sizeof(b)) != 0) ++g->buf_gen;  // new layout of the mask rows
  s->mbox = b;
  {
    ProfScope ps(g, P_MASKS);
    CK(launch_masks(g, *s, b, s->d_mask));
  }
  if (g->count_on) {
    // (offset, word) pairs, and the supercover voxel terms they OR together
    const unsigned long long words = (unsigned long long)b.words();
    g->h_counters[kCounters * P_MASKS + 0] += (unsigned long long)s->host.off.size() * words;
    g->h_counters[kCounters * P_MASKS + 1] += (unsigned long long)s->host.sc.size() * words;
  }
  s->mask_version = g->version;
  return IK_OK;
}

// Word box of the voxels within `reach` of `root` along every axis (the
// positions a joint reached through segments of that summed reach can take),
// clipped to the grid; the whole grid when root is outside it.
MaskBox reach_box(const Dims& d, const int32_t* root, int reach) {
  MaskBox b{0, 0, 0, d.wx - 1, d.ny - 1, d.nz - 1};
  if (!root || root[0] < 0 || root[0] >= d.nx || root[1] < 0 || root[1] >= d.ny || root[2] < 0 ||
      root[2] >= d.nz)
    return b;
  b.wx0 = std::max(0, root[0] - reach) >> 5;
  b.wx1 = std::min(d.nx - 1, root[0] + reach) >> 5;
  b.y0 = std::max(0, root[1] - reach);
  b.y1 = std::min(d.ny - 1, root[1] + reach);
  b.z0 = std::max(0, root[2] - reach);
  b.z1 = std::min(d.nz - 1, root[2] + reach);
  return b;
}

// Device tables of an arm for chains rooted at `root` (host pointer).  Every
// edge-mask word a kernel reads for segment k lies at a joint position that
// segments 1..k can reach from the root, so segment k's masks need only the
// word box of the root grown by the summed reach of segments 1..k.  root
// nullptr: the caller reads no edge masks (none are built).
std::vector<int32_t> arm_key(const ik_arm* arm) {
  std::vector<int32_t> k(arm->len, arm->len + arm->n_seg);
  int32_t tb;
  memcpy(&tb, &arm->tol, 4);
  k.push_back(tb);
  return k;
}

const std::vector<ik_cone>* arm_limits(ik_grid g, const ik_arm* arm) {
  auto it = g->limits.find(arm_key(arm));
  return it == g->limits.end() ? nullptr : &it->second;
}

bool has_axis(const ik_cone& c) { return c.axis[0] != 0 || c.axis[1] != 0 || c.axis[2] != 0; }

void fill_seg(const ShellDev* s, const ik_grid g, bool masks, SegDev* sd) {
  sd->off = s->d_off;
  sd->rows = s->d_rows;
  sd->tab = s->d_tab;
  sd->tabw = s->d_tabw;
  sd->tabr = s->d_tabr;
  sd->rowsr = s->d_rowsr;
  sd->sctab = s->d_sctab;
  sd->sc_start = s->d_sc_start;
  sd->sc = s->d_sc;
  sd->mask = masks ? s->d_mask : nullptr;
  sd->mbox = s->mbox;
  sd->occ = g->d_occ;
  sd->n = (int)s->host.off.size();
  sd->lo2 = s->host.lo2;
  sd->hi2 = s->host.hi2;
  sd->R = s->reach;
}

// Device tables of an arm for chains rooted at `root` (host pointer).  Every
// edge-mask word a kernel reads for segment k lies at a joint position that
// segments 1..k can reach from the root, so segment k's masks need only the
// word box of the root grown by the summed reach of segments 1..k.  root
// nullptr: the caller reads no edge masks (none are built).  A segment with
// a direction limit (ik_set_segment_limits) gets the cone's part of its
// shell, and the mirrored cone for the forward gathers.  used (nullable)
// receives every table whose edge masks the arm reads.
int resolve_arm(ik_grid g, const ik_arm* arm, const int32_t* root, ArmDev* ad,
                std::vector<std::pair<int, int>>* key, std::vector<ShellDev*>* used = nullptr) {
  int rc = check_arm(arm);
  if (rc) return rc;
  memset(ad, 0, sizeof(*ad));
  ad->S = arm->n_seg;
  if (key) key->clear();
  if (used) used->clear();
  const bool masks = g->use_masks && root;
  const std::vector<ik_cone>* lim = arm_limits(g, arm);
  ShellDev *sa[IK_MAX_SEG], *sf[IK_MAX_SEG];
  int reach = 0;
  for (int k = 0; k < arm->n_seg; ++k) {
    int lo2, hi2;
    shell_bounds(arm->len[k], (double)arm->tol, &lo2, &hi2);
    if (hi2 < lo2) return IK_ERR_ARG;
    ShellDev* whole = nullptr;
    rc = get_shell(g, lo2, hi2, &whole);
    if (rc) return rc;
    reach += whole->reach;
    sa[k] = sf[k] = whole;
    if (lim && has_axis((*lim)[k])) {
      ik_cone neg = (*lim)[k];
      for (int i = 0; i < 3; ++i) neg.axis[i] = -neg.axis[i];
      if ((rc = get_cone_shell(g, lo2, hi2, (*lim)[k], &sa[k]))) return rc;
      if ((rc = get_cone_shell(g, lo2, hi2, neg, &sf[k]))) return rc;
    }
    if (key) key->push_back(std::make_pair(lo2, hi2));
  }
  // masks once every table is known (a table shared by two segments may
  // grow its box for the second), then the device views
  reach = 0;
  for (int k = 0; k < arm->n_seg; ++k) {
    reach += sa[k]->reach;
    for (ShellDev* s : {sa[k], sf[k]}) {
      if (masks && (rc = ensure_masks(g, s, reach_box(g->d, root, reach)))) return rc;
      if (used && std::find(used->begin(), used->end(), s) == used->end()) used->push_back(s);
    }
  }
  for (int k = 0; k < arm->n_seg; ++k) {
    fill_seg(sa[k], g, masks, &ad->seg[k]);
    fill_seg(sf[k], g, masks, &ad->segf[k]);
    ad->len[k] = arm->len[k];
  }
  return IK_OK;
}

bool point_inside(const Dims& d, const int32_t* p) {
  return p[0] >= 0 && p[1] >= 0 && p[2] >= 0 && p[0] < d.nx && p[1] < d.ny && p[2] < d.nz;
}

// Forward sets F_0..F_S for `root` (host int[3]), cached.
int ensure_forward(ik_grid g, const ArmDev& ad, const std::vector<std::pair<int, int>>& key,
                   const int32_t* root) {
  if (g->f_valid && g->f_version == g->version && g->f_key == key && g->f_root[0] == root[0] &&
      g->f_root[1] == root[1] && g->f_root[2] == root[2])
    return IK_OK;
  g->f_valid = false;
  const Dims& d = g->d;
  const int S = ad.S;
  int rc = ensure(g, g->F, (size_t)(S + 1) * d.nw * 4);
  if (rc) return rc;
  if ((rc = ensure(g, g->F_box, (size_t)(S + 1) * 24))) return rc;
  rc = to_device(g, g->b_root, root, 12);
  if (rc) return rc;
  uint32_t* F = ptr<uint32_t>(g->F);
  int32_t* fb = ptr<int32_t>(g->F_box);
  CK(cudaMemsetAsync(fb, kBoxEmptyByte, (size_t)(S + 1) * 24, g->st));
  {
    ProfScope ps(g, P_SEED);
    CK(launch_seed_points(d, ptr<int32_t>(g->b_root), 1, nullptr, g->d_occ, F, d.nw, nullptr, fb, 0,
                          g->st));
  }
  for (int k = 1; k <= S; ++k) {
    ProfScope ps(g, P_FWD);
    CK(launch_propagate(d, g->tc, ad.segf[k - 1], F + (k - 1) * d.nw, 0, nullptr, 0, g->d_occ, F + k * d.nw,
                        0, 1, fb + 6 * (k - 1), fb + 6 * k, 0, g->st, counters(g, P_FWD)));
  }
  g->f_valid = true;
  g->f_version = g->version;
  g->f_key = key;
  memcpy(g->f_root, root, 12);
  return IK_OK;
}

// Backward pass for Q queries whose last set (index S) is already seeded in
// V (query stride (S+1) * nw): V_{k-1} = F_{k-1} & D_k(V_k) for k = S..1.
int backward_sets(ik_grid g, const ArmDev& ad, uint32_t* V, int Q, int prof_id, int32_t* box) {
  const Dims& d = g->d;
  const int S = ad.S;
  const long qs = (long)(S + 1) * d.nw;
  const uint32_t* F = ptr<uint32_t>(g->F);
  const int32_t* fb = ptr<int32_t>(g->F_box);
  // work list scratch: every (query, tile) pair at most, and the count
  WorkList wl{};
  const WorkList* wlp = nullptr;
  if (Q >= kListMinQueries && g->work_list > 0) {
    const long cap = (long)Q * g->tc.tiles_y * g->tc.tiles_z;
    int rc = ensure(g, g->b_list, (size_t)cap * sizeof(int2) + 16);
    if (rc) return rc;
    wl.items = ptr<int2>(g->b_list);
    wl.count = reinterpret_cast<int*>(wl.items + cap);
    wl.cap = cap;
    wl.blocks = g->num_sms * 4;  // about as many as stay resident
    wlp = &wl;
  }
  // R_1 + ... + R_k for the bound of each level's output below
  int rsum[IK_MAX_SEG + 1] = {0};
  for (int k = 1; k <= S; ++k) rsum[k] = rsum[k - 1] + ad.seg[k - 1].R;
  for (int k = S; k >= 1; --k) {
    // V_{k-1} lies within R_1 + ... + R_{k-1} of the root (it is inside
    // F_{k-1}) and, for a point target, within R_k + ... + R_S of it. The
    // work list pays where that bound leaves at most an eighth of the tiles
    // (the levels next to either end of the arm); on the others the plain
    // grid of every (tile, query) was measured faster. Either form gives the
    // same sets.
    const WorkList* wk = nullptr;
    if (wlp && g->work_list == 2) {
      wk = wlp;
    } else if (wlp) {
      const TileCfg& tc = g->tc;
      const int rf = rsum[k - 1], rt = rsum[S] - rsum[k - 1];
      auto span = [&](int c, int n) {
        const int lo = std::max(0, c - rf), hi = std::min(n - 1, c + rf);
        return std::max(0, std::min(hi - lo + 1, 2 * rt + 1));
      };
      const long ty = std::min(tc.tiles_y, (span(g->f_root[1], d.ny) + tc.TY - 1) / tc.TY + 1);
      const long tz = std::min(tc.tiles_z, (span(g->f_root[2], d.nz) + tc.TZ - 1) / tc.TZ + 1);
      // with row lanes (which skip rows whose source windows are empty) the
      // full grid pays down to sparser levels: the list then takes only the
      // levels at most a 16th of whose tiles can be live (on the 128^3 step,
      // levels 1 and 8; levels 2 and 7 measured faster on the full grid)
      const bool rows = tc.rows && g->use_masks && (d.wx == 1 || d.wx == 2 || d.wx == 4) && ad.seg[k - 1].R <= 31;
      if ((rows ? 16 : 8) * ty * tz <= (long)tc.tiles_y * tc.tiles_z) wk = wlp;
    }
    const SegDev& seg = ad.seg[k - 1];
    if (propagate_listed(g->tc, seg, Q, qs, wk)) {
      ProfScope pt(g, P_TILE_LIST);
      CK(launch_tile_list(d, g->tc, seg.R, Q, box + 6 * k, 6L * (S + 1), fb + 6 * (k - 1),
                          V + (long)(k - 1) * d.nw, qs, *wk, g->st));
    } else {
      wk = nullptr;
    }
    ProfScope ps(g, prof_id);
    // the waypoint pass is also recorded per level (work counters go there)
    ProfScope pl(g, prof_id == P_BWD_WAY ? P_WAY_K1 + k - 1 : -1);
    unsigned long long* cnt = counters(g, prof_id == P_BWD_WAY ? P_WAY_K1 + k - 1 : prof_id);
    CK(launch_propagate(d, g->tc, seg, V + (long)k * d.nw, qs, F + (long)(k - 1) * d.nw, 0, g->d_occ,
                        V + (long)(k - 1) * d.nw, qs, Q, box + 6 * k, box + 6 * (k - 1), 6L * (S + 1),
                        g->st, cnt, wk));
  }
  return IK_OK;
}

int copy_out(ik_grid g, void* dst, const void* src, size_t bytes, int on_device) {
  if (!dst || bytes == 0) return IK_OK;
  CK(cudaMemcpyAsync(dst, src, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                     g->st));
  return IK_OK;
}

int sync(ik_grid g) {
  CK(cudaStreamSynchronize(g->st));
  CK(cudaGetLastError());
  return IK_OK;
}

int set_device(ik_grid g) {
  if (!g) return IK_ERR_ARG;
  CK(cudaSetDevice(g->device));
  return IK_OK;
}


}  // namespace

extern "C" {

int ik_version(void) { return 1; }

const char* ik_strerror(int code) {
  switch (code) {
    case IK_OK: return "ok";
    case IK_ERR_ARG: return "invalid argument";
    case IK_ERR_OOM: return "out of memory";
    case IK_ERR_CUDA: return "CUDA error";
    case IK_ERR_TIMEOUT: return "device wait timed out";
    case IK_ERR_STATE: return "invalid state";
    case IK_ERR_UNSUPPORTED: return "unsupported request";
    default: return "unknown error";
  }
}

const char* ik_last_error_message(void) { return g_last_error.c_str(); }

int ik_create_grid(int nx, int ny, int nz, void* cuda_stream, ik_grid* out) {
  if (!out) return IK_ERR_ARG;
  *out = nullptr;
  if (nx < 32 || nx > 1024 || nx % 32 != 0 || ny < 1 || ny > 1024 || nz < 1 || nz > 1024)
    return IK_ERR_ARG;
  ik_grid g = new ik_grid_s();
  cudaError_t e = cudaGetDevice(&g->device);
  if (e != cudaSuccess) {
    delete g;
    return fail_cuda(e);
  }
  g->d.nx = nx;
  g->d.ny = ny;
  g->d.nz = nz;
  g->d.wx = nx / 32;
  g->d.nw = (long)g->d.wx * ny * nz;
  g->tc = make_tile_cfg(g->d);
  g->st = (cudaStream_t)cuda_stream;
  {
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, g->device) == cudaSuccess && sms > 0)
      g->num_sms = sms;
  }
  e = set_kernel_attributes();
  if (e == cudaSuccess) e = cudaMalloc(&g->d_occ, g->d.nw * 4);
  if (e == cudaSuccess) e = cudaMalloc(&g->d_occ_raw, g->d.nw * 4);
  if (e == cudaSuccess) e = cudaMalloc(&g->d_tma_slow, sizeof(int));
  if (e == cudaSuccess) e = cudaMemsetAsync(g->d_tma_slow, 0, sizeof(int), g->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(g->d_occ, 0, g->d.nw * 4, g->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(g->d_occ_raw, 0, g->d.nw * 4, g->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(g->st);
  if (e != cudaSuccess) {
    cudaFree(g->d_occ);
    cudaFree(g->d_occ_raw);
    delete g;
    return fail_cuda(e);
  }
  *out = g;
  return IK_OK;
}

int ik_destroy_grid(ik_grid g) {
  if (!g) return IK_ERR_ARG;
  cudaSetDevice(g->device);
  cudaStreamSynchronize(g->st);
  std::vector<ShellDev*> all;
  for (auto& kv : g->shells) all.push_back(kv.second);
  for (auto& kv : g->cone_shells) all.push_back(kv.second);
  for (ShellDev* s : all) {
    cudaFree(s->d_off);
    cudaFree(s->d_tab);
    cudaFree(s->d_sctab);
    cudaFree(s->d_sctab_tma);
    cudaFree(s->d_tabw);
    cudaFree(s->d_tabr);
    cudaFree(s->d_rowsr);
    cudaFree(s->d_sctabr);
    cudaFree(s->d_rows);
    cudaFree(s->d_sc_start);
    cudaFree(s->d_sc);
    cudaFree(s->d_mask);
    delete s;
  }
  cudaFree(g->d_tma_slow);
  DevBuf* bufs[] = {&g->F, &g->V, &g->Vw, &g->chain, &g->boxes, &g->F_box, &g->V_box, &g->Vw_box,
                    &g->b_rp, &g->b_rin, &g->b_rc, &g->b_root, &g->b_targets,
                    &g->b_reach, &g->b_found, &g->b_poses, &g->b_relax, &g->b_status, &g->b_eps,
                    &g->b_g, &g->b_valid, &g->b_old, &g->b_list, &g->b_tposes, &g->b_fold};
  for (DevBuf* b : bufs) cudaFree(b->p);
  for (void* p : g->retired) cudaFree(p);
  for (cudaEvent_t e : g->ev_pool) cudaEventDestroy(e);
  cudaFree(g->d_counters);
  cudaFree(g->d_occ);
  cudaFree(g->d_occ_raw);
  delete g;
  return IK_OK;
}

size_t ik_grid_words(ik_grid g) { return g ? (size_t)g->d.nw : 0; }

// d_occ from d_occ_raw: dilated by the ball |v|^2 <= dilate_r2, or a copy.
static int apply_dilation(ik_grid g) {
  if (g->dilate_r2 > 0)
    CK(launch_dilate(g->d, g->d_occ_raw, g->dilate_r2, g->d_occ, g->st));
  else
    CK(cudaMemcpyAsync(g->d_occ, g->d_occ_raw, (size_t)g->d.nw * 4, cudaMemcpyDeviceToDevice, g->st));
  return IK_OK;
}

int ik_set_obstacles(ik_grid g, const uint32_t* occ_words, size_t n_words, int on_device) {
  int rc = set_device(g);
  if (rc) return rc;
  if (!occ_words || n_words != (size_t)g->d.nw) return IK_ERR_ARG;
  CK(cudaMemcpyAsync(g->d_occ_raw, occ_words, n_words * 4,
                     on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, g->st));
  if ((rc = apply_dilation(g))) return rc;
  ++g->version;
  return sync(g);
}

int ik_set_boxes(ik_grid g, const int32_t* boxes, int n_boxes, int on_device) {
  int rc = set_device(g);
  if (rc) return rc;
  if (n_boxes < 0 || (n_boxes > 0 && !boxes)) return IK_ERR_ARG;
  const int32_t* db = boxes;
  if (n_boxes > 0 && !on_device) {
    rc = to_device(g, g->boxes, boxes, (size_t)n_boxes * 24);
    if (rc) return rc;
    db = ptr<int32_t>(g->boxes);
  }
  {
    ProfScope ps(g, P_RASTER);
    CK(launch_rasterize(g->d, db, n_boxes, g->d_occ_raw, g->st));
    if ((rc = apply_dilation(g))) return rc;
  }
  ++g->version;
  return sync(g);
}

int ik_get_obstacles(ik_grid g, uint32_t* occ_words, size_t n_words, int on_device) {
  int rc = set_device(g);
  if (rc) return rc;
  if (!occ_words || n_words != (size_t)g->d.nw) return IK_ERR_ARG;
  rc = copy_out(g, occ_words, g->d_occ, n_words * 4, on_device);
  if (rc) return rc;
  return sync(g);
}

int ik_forward_sets(ik_grid g, const ik_arm* arm, const int32_t root[3], uint32_t* fsets_out,
                    int on_device) {
  int rc = set_device(g);
  if (rc) return rc;
  if (!root || !point_inside(g->d, root)) return IK_ERR_ARG;
  ArmDev ad;
  std::vector<std::pair<int, int>> key;
  if ((rc = resolve_arm(g, arm, root, &ad, &key))) return rc;
  if ((rc = ensure_forward(g, ad, key, root))) return rc;
  if ((rc = copy_out(g, fsets_out, g->F.p, (size_t)(ad.S + 1) * g->d.nw * 4, on_device))) return rc;
  return sync(g);
}

// Reach for n targets; every array is a device pointer when on_device.
// Reach for n targets (or, with d_tset, for the one target set d_tset).
// `ad` grows the forward sets; `adb` (nullable: ad) runs the backward sets
// and the traceback, so that it may restrict the last segment to a cone.
static int reach_many_impl(ik_grid g, const ArmDev& ad, const std::vector<std::pair<int, int>>& key,
                           const int32_t* root, const int32_t* targets, int n, int32_t* poses_out,
                           int32_t* found_out, uint32_t* vsets_out, int on_device,
                           int32_t** d_poses, int32_t** d_found, const ArmDev* adb = nullptr,
                           const uint32_t* d_tset = nullptr) {
  const Dims& d = g->d;
  const int S = ad.S;
  const ArmDev& ab = adb ? *adb : ad;
  int rc = ensure_forward(g, ad, key, root);
  if (rc) return rc;
  const long qs = (long)(S + 1) * d.nw;
  if ((rc = ensure(g, g->V, (size_t)n * qs * 4))) return rc;
  uint32_t* V = ptr<uint32_t>(g->V);
  const int32_t* dt = targets;
  if (!on_device && !d_tset) {
    if ((rc = to_device(g, g->b_targets, targets, (size_t)n * 12))) return rc;
    dt = ptr<int32_t>(g->b_targets);
  }
  if ((rc = to_device(g, g->b_root, root, 12))) return rc;
  if ((rc = ensure(g, g->V_box, (size_t)n * (S + 1) * 24))) return rc;
  int32_t* vb = ptr<int32_t>(g->V_box);
  CK(cudaMemsetAsync(vb, kBoxEmptyByte, (size_t)n * (S + 1) * 24, g->st));
  const uint32_t* F = ptr<uint32_t>(g->F);
  {
    ProfScope ps(g, P_SEED);
    if (d_tset)
      CK(launch_seed_set(d, d_tset, F + (long)S * d.nw, V + (long)S * d.nw, vb + 6 * S, g->st));
    else
      CK(launch_seed_points(d, dt, n, F + (long)S * d.nw, nullptr, V + (long)S * d.nw, qs, nullptr,
                            vb + 6 * S, 6L * (S + 1), g->st));
  }
  if ((rc = backward_sets(g, ab, V, n, P_BWD_REACH, vb))) return rc;
  int32_t* dp = poses_out;
  int32_t* df = found_out;
  if (!on_device || !poses_out || !found_out) {
    if ((rc = ensure(g, g->b_reach, (size_t)n * 12 * (S + 1)))) return rc;
    if ((rc = ensure(g, g->b_found, (size_t)n * 4))) return rc;
    dp = ptr<int32_t>(g->b_reach);
    df = ptr<int32_t>(g->b_found);
  }
  {
    ProfScope ps(g, P_TRACE);
    CK(launch_traceback(d, ab, ptr<int32_t>(g->b_root), V, qs, n, dp, df, g->st));
  }
  if (!on_device) {
    if ((rc = copy_out(g, poses_out, dp, (size_t)n * 12 * (S + 1), 0))) return rc;
    if ((rc = copy_out(g, found_out, df, (size_t)n * 4, 0))) return rc;
  }
  if (vsets_out && (rc = copy_out(g, vsets_out, V, (size_t)n * qs * 4, on_device))) return rc;
  if (d_poses) *d_poses = dp;
  if (d_found) *d_found = df;
  return IK_OK;
}

int ik_solve_reach_many(ik_grid g, const ik_arm* arm, const int32_t root[3], const int32_t* targets,
                        int n, int32_t* poses_out, int32_t* found_out, uint32_t* vsets_out,
                        int on_device) {
  int rc = set_device(g);
  if (rc) return rc;
  if (!root || !point_inside(g->d, root) || n < 0 || (n > 0 && !targets)) return IK_ERR_ARG;
  if (n == 0) return IK_OK;
  if (!on_device) {
    for (int i = 0; i < n; ++i)
      if (!point_inside(g->d, targets + 3 * i)) return IK_ERR_ARG;
  }
  ArmDev ad;
  std::vector<std::pair<int, int>> key;
  if ((rc = resolve_arm(g, arm, root, &ad, &key))) return rc;
  if ((rc = reach_many_impl(g, ad, key, root, targets, n, poses_out, found_out, vsets_out, on_device,
                            nullptr, nullptr)))
    return rc;
  return sync(g);
}

// The arm with its last segment restricted to `cone` (tables and edge masks
// of the cone's part of the shell, over the reachable box of the root).
static int cone_arm(ik_grid g, const ik_arm* arm, const ik_cone* cone, const int32_t* root,
                    const ArmDev& ad, ArmDev* adc) {
  *adc = ad;
  const int S = ad.S;
  // an approach cone replaces the last segment's table: with a direction
  // limit on that segment as well the two would have to be intersected
  const std::vector<ik_cone>* lim = arm_limits(g, arm);
  if (lim && has_axis((*lim)[S - 1])) return IK_ERR_ARG;
  ShellDev* s = nullptr;
  int rc = get_cone_shell(g, ad.seg[S - 1].lo2, ad.seg[S - 1].hi2, *cone, &s);
  if (rc) return rc;
  int reach = 0;
  for (int k = 0; k < S; ++k) reach += ad.seg[k].R;
  const bool masks = g->use_masks;
  if (masks && (rc = ensure_masks(g, s, reach_box(g->d, root, reach)))) return rc;
  SegDev& sd = adc->seg[S - 1];
  sd.off = s->d_off;
  sd.rows = s->d_rows;
  sd.tab = s->d_tab;
  sd.tabw = s->d_tabw;
  sd.tabr = s->d_tabr;
  sd.rowsr = s->d_rowsr;
  sd.sctab = s->d_sctab;
  sd.sc_start = s->d_sc_start;
  sd.sc = s->d_sc;
  sd.mask = masks ? s->d_mask : nullptr;
  sd.mbox = s->mbox;
  sd.n = (int)s->host.off.size();
  sd.R = s->reach;
  return IK_OK;
}

int ik_set_segment_limits(ik_grid g, const ik_arm* arm, const ik_cone* limits) {
  int rc = set_device(g);
  if (rc) return rc;
  if ((rc = check_arm(arm))) return rc;
  const std::vector<int32_t> key = arm_key(arm);
  bool any = false;
  if (limits) {
    for (int k = 0; k < arm->n_seg; ++k) {
      if (!has_axis(limits[k])) continue;
      if ((rc = check_cone(&limits[k]))) return rc;
      any = true;
    }
  }
  if (any)
    g->limits[key] = std::vector<ik_cone>(limits, limits + arm->n_seg);
  else
    g->limits.erase(key);
  g->f_valid = false;  // cached forward sets may be of the old limits
  return IK_OK;
}

int ik_solve_reach_many_cone(ik_grid g, const ik_arm* arm, const ik_cone* cone, const int32_t root[3],
                             const int32_t* targets, int n, int32_t* poses_out, int32_t* found_out,
                             uint32_t* vsets_out, int on_device) {
  int rc = set_device(g);
  if (rc) return rc;
  if (!root || !point_inside(g->d, root) || n < 0 || (n > 0 && !targets)) return IK_ERR_ARG;
  if ((rc = check_cone(cone))) return rc;
  if (n == 0) return IK_OK;
  if (!on_device) {
    for (int i = 0; i < n; ++i)
      if (!point_inside(g->d, targets + 3 * i)) return IK_ERR_ARG;
  }
  ArmDev ad, adc;
  std::vector<std::pair<int, int>> key;
  if ((rc = resolve_arm(g, arm, root, &ad, &key))) return rc;
  if (cone) {
    // the cone's table may be one of the arm's (a segment limit with the
    // same cone): resolve the arm again once its masks are in place
    if ((rc = cone_arm(g, arm, cone, root, ad, &adc))) return rc;
    if ((rc = resolve_arm(g, arm, root, &ad, &key))) return rc;
    if ((rc = cone_arm(g, arm, cone, root, ad, &adc))) return rc;
  }
  if ((rc = reach_many_impl(g, ad, key, root, targets, n, poses_out, found_out, vsets_out, on_device,
                            nullptr, nullptr, cone ? &adc : nullptr)))
    return rc;
  return sync(g);
}

int ik_solve_reach_set(ik_grid g, const ik_arm* arm, const ik_cone* cone, const int32_t root[3],
                       const uint32_t* target_words, int32_t* pose_out, uint32_t* vsets_out,
                       int* found) {
  int rc = set_device(g);
  if (rc) return rc;
  if (!root || !point_inside(g->d, root) || !target_words || !pose_out || !found) return IK_ERR_ARG;
  if ((rc = check_cone(cone))) return rc;
  ArmDev ad, adc;
  std::vector<std::pair<int, int>> key;
  if ((rc = resolve_arm(g, arm, root, &ad, &key))) return rc;
  if (cone) {
    if ((rc = cone_arm(g, arm, cone, root, ad, &adc))) return rc;
    if ((rc = resolve_arm(g, arm, root, &ad, &key))) return rc;
    if ((rc = cone_arm(g, arm, cone, root, ad, &adc))) return rc;
  }
  if ((rc = to_device(g, g->b_old, target_words, (size_t)g->d.nw * 4))) return rc;
  int32_t fnd = 0;
  if ((rc = reach_many_impl(g, ad, key, root, nullptr, 1, pose_out, &fnd, vsets_out, 0, nullptr, nullptr,
                            cone ? &adc : nullptr, ptr<uint32_t>(g->b_old))))
    return rc;
  if ((rc = sync(g))) return rc;
  *found = fnd;
  return IK_OK;
}

int ik_solve_reach(ik_grid g, const ik_arm* arm, const int32_t root[3], const int32_t target[3],
                   int32_t* pose_out, uint32_t* vsets_out, int* found) {
  if (!pose_out || !found || !target) return IK_ERR_ARG;
  int32_t f = 0;
  int rc = ik_solve_reach_many(g, arm, root, target, 1, pose_out, &f, vsets_out, 0);
  *found = f;
  return rc;
}

int ik_guide(ik_grid g, const ik_arm* arm, const int32_t* reach_pose, int n_way, int32_t* g_out) {
  int rc = set_device(g);
  if (rc) return rc;
  if (!reach_pose || !g_out || n_way < 2) return IK_ERR_ARG;
  if ((rc = check_arm(arm))) return rc;
  ArmDev ad;
  memset(&ad, 0, sizeof(ad));
  ad.S = arm->n_seg;
  for (int k = 0; k < ad.S; ++k) ad.len[k] = arm->len[k];
  const int S = ad.S;
  if ((rc = to_device(g, g->b_reach, reach_pose, (size_t)12 * (S + 1)))) return rc;
  if ((rc = ensure(g, g->b_g, (size_t)12 * n_way))) return rc;
  if ((rc = ensure(g, g->b_eps, (size_t)4 * n_way))) return rc;
  CK(launch_guide_targets(g->d, ad, g->d_occ, nullptr, ptr<int32_t>(g->b_reach), nullptr, 1, n_way, 0,
                          0, 0, ptr<int32_t>(g->b_g), ptr<int32_t>(g->b_eps), nullptr, nullptr,
                          g->st));
  if ((rc = copy_out(g, g_out, g->b_g.p, (size_t)12 * n_way, 0))) return rc;
  return sync(g);
}

// Survivor sets of P paths x W waypoints (waypoints j >= j_lo) whose reach
// poses are on the device (d_reach [P][S+1][3], d_found nullable).
static int waypoint_sets_impl(ik_grid g, const ArmDev& ad, const int32_t* d_reach,
                              const int32_t* d_found, int P, int W, int j_lo, int eps2,
                              int eps2_max, const int32_t* c_arr = nullptr,
                              const GuideArm* ga = nullptr, int32_t* fold_at = nullptr) {
  const Dims& d = g->d;
  const int S = ad.S;
  const long qs = (long)(S + 1) * d.nw;
  int rc = ensure(g, g->Vw, (size_t)P * W * qs * 4);
  if (rc) return rc;
  if ((rc = ensure(g, g->b_g, (size_t)12 * P * W))) return rc;
  if ((rc = ensure(g, g->b_eps, (size_t)4 * P * W))) return rc;
  uint32_t* Vw = ptr<uint32_t>(g->Vw);
  if ((rc = ensure(g, g->Vw_box, (size_t)P * W * (S + 1) * 24))) return rc;
  int32_t* wb = ptr<int32_t>(g->Vw_box);
  CK(cudaMemsetAsync(wb, kBoxEmptyByte, (size_t)P * W * (S + 1) * 24, g->st));
  // zero the seeded (last) set of every waypoint
  CK(cudaMemset2DAsync(Vw + (long)S * d.nw, (size_t)qs * 4, 0, (size_t)d.nw * 4, (size_t)P * W, g->st));
  const uint32_t* F = ptr<uint32_t>(g->F);
  {
    ProfScope ps(g, P_GUIDE);
    CK(launch_guide_targets(d, ad, g->d_occ, F + (long)S * d.nw, d_reach, d_found, P, W, j_lo, eps2,
                            eps2_max, ptr<int32_t>(g->b_g), ptr<int32_t>(g->b_eps), Vw, wb, g->st,
                            c_arr, ga, fold_at));
  }
  if (j_lo == 0) return backward_sets(g, ad, Vw, P * W, P_BWD_WAY, wb);
  // only waypoints j >= j_lo (P == 1 in that case)
  for (int p = 0; p < P; ++p)
    if ((rc = backward_sets(g, ad, Vw + ((long)p * W + j_lo) * qs, W - j_lo, P_BWD_WAY,
                            wb + ((long)p * W + j_lo) * (S + 1) * 6)))
      return rc;
  return IK_OK;
}

static int check_path_params(const ik_path_params* pp) {
  if (!pp || pp->n_way < 2 || pp->n_way > 4096 || pp->delta < 0 || pp->delta > 4096 ||
      pp->eps2 < 0 || pp->eps2 > 4096 || pp->eps2_max < 0 || pp->eps2_max > 4096 ||
      pp->max_relax < -1)
    return IK_ERR_ARG;
  return IK_OK;
}

int ik_waypoint_sets(ik_grid g, const ik_arm* arm, const int32_t* reach_pose, int n_way, int eps2,
                     int eps2_max, int32_t* eps2_used, uint32_t* vsets_out) {
  int rc = set_device(g);
  if (rc) return rc;
  if (!reach_pose || n_way < 2 || n_way > 4096 || eps2 < 0 || eps2 > 4096 || eps2_max < 0 ||
      eps2_max > 4096)
    return IK_ERR_ARG;
  ArmDev ad;
  std::vector<std::pair<int, int>> key;
  if ((rc = resolve_arm(g, arm, reach_pose, &ad, &key))) return rc;
  const int S = ad.S;
  for (int k = 0; k <= S; ++k)
    if (!point_inside(g->d, reach_pose + 3 * k)) return IK_ERR_ARG;
  if ((rc = ensure_forward(g, ad, key, reach_pose))) return rc;
  if ((rc = to_device(g, g->b_reach, reach_pose, (size_t)12 * (S + 1)))) return rc;
  if ((rc = waypoint_sets_impl(g, ad, ptr<int32_t>(g->b_reach), nullptr, 1, n_way, 0, eps2, eps2_max)))
    return rc;
  if ((rc = copy_out(g, eps2_used, g->b_eps.p, (size_t)4 * n_way, 0))) return rc;
  if ((rc = copy_out(g, vsets_out, g->Vw.p, (size_t)n_way * (S + 1) * g->d.nw * 4, 0))) return rc;
  return sync(g);
}

// Smooth chains for P paths whose waypoint survivor sets are in g->Vw and
// whose preset poses are in d_poses.
static int chain_impl(ik_grid g, const ArmDev& ad, const ik_path_params* pp, int P, int mode, int c,
                      const int32_t* d_found, int32_t* d_poses, int32_t* d_relax, int32_t* d_status,
                      const int32_t* c_arr = nullptr, const int32_t* rad = nullptr) {
  const Dims& d = g->d;
  const int S = ad.S;
  int rc = ensure(g, g->chain, (size_t)P * 2 * (S + 1) * d.nw * 4, true);
  if (rc) return rc;
  ChainArgs a;
  a.P = P;
  a.W = pp->n_way;
  a.c = c;
  a.mode = mode;
  a.delta = pp->delta;
  a.max_relax = pp->max_relax;
  a.found = d_found;
  a.Vw = ptr<uint32_t>(g->Vw);
  a.eps_used = ptr<int32_t>(g->b_eps);
  a.poses = d_poses;
  a.relax = d_relax;
  a.status = d_status;
  a.scratch = ptr<uint32_t>(g->chain);
  a.relaxed_eps_base = pp->eps2;
  a.c_arr = c_arr;
  // the given radius per joint, or delta for every joint
  a.per_joint = rad != nullptr;
  a.rad[0] = -1;
  for (int k = 1; k <= IK_MAX_SEG; ++k) a.rad[k] = (rad && k <= S) ? rad[k - 1] : pp->delta;
  a.vbox = ptr<int32_t>(g->Vw_box);
  a.counters = counters(g, P_CHAIN);
  {
    ProfScope ps(g, P_CHAIN);
    CK(launch_smooth_chain(d, ad, a, g->st));
  }
  return IK_OK;
}

static int validate_impl(ik_grid g, const ArmDev& ad, const int32_t* d_poses, int n, int32_t* d_valid) {
  {
    ProfScope ps(g, P_VALIDATE);
    CK(launch_validate(g->d, ad, g->d_occ, d_poses, n, d_valid, g->st));
  }
  return IK_OK;
}

int ik_validate_poses(ik_grid g, const ik_arm* arm, const int32_t* poses, int n, int32_t* valid_out) {
  int rc = set_device(g);
  if (rc) return rc;
  if (n < 0 || (n > 0 && (!poses || !valid_out))) return IK_ERR_ARG;
  if (n == 0) return IK_OK;
  ArmDev ad;
  if ((rc = resolve_arm(g, arm, nullptr, &ad, nullptr))) return rc;
  const int S = ad.S;
  if ((rc = to_device(g, g->b_poses, poses, (size_t)n * 12 * (S + 1)))) return rc;
  if ((rc = ensure(g, g->b_valid, (size_t)4 * n))) return rc;
  if ((rc = validate_impl(g, ad, ptr<int32_t>(g->b_poses), n, ptr<int32_t>(g->b_valid)))) return rc;
  if ((rc = copy_out(g, valid_out, g->b_valid.p, (size_t)4 * n, 0))) return rc;
  return sync(g);
}

int ik_plan_path(ik_grid g, const ik_arm* arm, const int32_t* reach_pose, const ik_path_params* pp,
                 int32_t* poses_out, int32_t* relax_out, int* status) {
  int rc = set_device(g);
  if (rc) return rc;
  if (!reach_pose || !poses_out || !relax_out || !status) return IK_ERR_ARG;
  if ((rc = check_path_params(pp))) return rc;
  ArmDev ad;
  std::vector<std::pair<int, int>> key;
  if ((rc = resolve_arm(g, arm, reach_pose, &ad, &key))) return rc;
  const int S = ad.S, W = pp->n_way;
  const size_t pose_bytes = (size_t)12 * (S + 1);
  // the reach pose must be a valid pose of this arm in this grid
  if ((rc = to_device(g, g->b_reach, reach_pose, pose_bytes))) return rc;
  if ((rc = ensure(g, g->b_valid, 4))) return rc;
  if ((rc = validate_impl(g, ad, ptr<int32_t>(g->b_reach), 1, ptr<int32_t>(g->b_valid)))) return rc;
  int32_t valid = 0;
  if ((rc = copy_out(g, &valid, g->b_valid.p, 4, 0))) return rc;
  if ((rc = sync(g))) return rc;
  if (!valid) {
    *status = IK_PATH_UNREACHABLE;
    return IK_OK;
  }
  if ((rc = ensure_forward(g, ad, key, reach_pose))) return rc;
  if ((rc = waypoint_sets_impl(g, ad, ptr<int32_t>(g->b_reach), nullptr, 1, W, 0, pp->eps2, pp->eps2_max)))
    return rc;
  if ((rc = ensure(g, g->b_poses, pose_bytes * W))) return rc;
  if ((rc = ensure(g, g->b_relax, (size_t)8 * W))) return rc;
  if ((rc = ensure(g, g->b_status, 4))) return rc;
  int32_t* dposes = ptr<int32_t>(g->b_poses);
  CK(cudaMemcpyAsync(dposes + (long)(W - 1) * 3 * (S + 1), g->b_reach.p, pose_bytes,
                     cudaMemcpyDeviceToDevice, g->st));
  if ((rc = chain_impl(g, ad, pp, 1, 0, 0, nullptr, dposes, ptr<int32_t>(g->b_relax),
                       ptr<int32_t>(g->b_status))))
    return rc;
  int32_t st = 0;
  if ((rc = copy_out(g, poses_out, dposes, pose_bytes * W, 0))) return rc;
  if ((rc = copy_out(g, relax_out, g->b_relax.p, (size_t)8 * W, 0))) return rc;
  if ((rc = copy_out(g, &st, g->b_status.p, 4, 0))) return rc;
  if ((rc = sync(g))) return rc;
  *status = st;
  return IK_OK;
}

int ik_plan_path_follow(ik_grid g, const ik_arm* arm, const int32_t* reach_pose, const ik_follow_params* fp,
                        int32_t* poses_out, int32_t* relax_out, int* status) {
  int rc = set_device(g);
  if (rc) return rc;
  if (!reach_pose || !poses_out || !relax_out || !status || !fp) return IK_ERR_ARG;
  if ((rc = check_arm(arm))) return rc;
  const int S = arm->n_seg, fold = fp->fold;
  const int F = S - (fold ? 1 : 0), n = fp->n_per_seg;
  if ((fold != 0 && fold != 1) || F < 1 || n < 1 || n > 64 || fp->eps2 < 0 || fp->eps2 > 4096 ||
      fp->eps2_max < 0 || fp->eps2_max > 4096 || fp->max_relax < -1)
    return IK_ERR_ARG;
  if (fp->paper_radii != 0 && fp->paper_radii != 1) return IK_ERR_ARG;
  int32_t rad[IK_MAX_SEG];
  if (fp->paper_radii) {
    // the paper's filter on joints 1 and 2 from the waypoint spacing
    int lmax = 0;
    for (int k = 0; k < F; ++k) lmax = std::max(lmax, (int)arm->len[k]);
    const int spacing = (lmax + n - 1) / n;
    for (int k = 0; k < IK_MAX_SEG; ++k) rad[k] = -1;
    rad[0] = (spacing + 1) / 2 + 1;
    if (F >= 2) rad[1] = spacing + 1;
  } else {
    for (int k = 0; k < IK_MAX_SEG; ++k) rad[k] = fp->radius[k];
  }
  for (int k = 0; k < F; ++k)
    if (rad[k] < -1 || rad[k] > 4096) return IK_ERR_ARG;
  const int W = F * n + 1;
  if (W > 4096) return IK_ERR_ARG;
  // the paper's form has no direction limits: an arm with limits is refused
  if (arm_limits(g, arm)) return IK_ERR_UNSUPPORTED;
  ArmDev ad;
  std::vector<std::pair<int, int>> key;
  if ((rc = resolve_arm(g, arm, reach_pose, &ad, &key))) return rc;
  const size_t pose_bytes = (size_t)12 * (S + 1), tpose_bytes = (size_t)12 * (F + 1);
  // the reach pose must be a valid pose of this arm in this grid
  if ((rc = to_device(g, g->b_reach, reach_pose, pose_bytes))) return rc;
  if ((rc = ensure(g, g->b_valid, 4))) return rc;
  if ((rc = validate_impl(g, ad, ptr<int32_t>(g->b_reach), 1, ptr<int32_t>(g->b_valid)))) return rc;
  int32_t valid = 0;
  if ((rc = copy_out(g, &valid, g->b_valid.p, 4, 0))) return rc;
  if ((rc = sync(g))) return rc;
  if (!valid) {
    *status = IK_PATH_UNREACHABLE;
    return IK_OK;
  }
  // the follower's arm: the first F segments (their device tables as resolved)
  ArmDev af = ad;
  af.S = F;
  std::vector<std::pair<int, int>> keyF(key.begin(), key.begin() + F);
  if ((rc = ensure_forward(g, af, keyF, reach_pose))) return rc;
  GuideArm ga;
  ga.S = F;
  for (int k = 0; k < S; ++k) ga.len[k] = arm->len[k];
  ga.n_per_seg = n;
  ga.pose_joints = S + 1;
  ga.fold_len = fold ? arm->len[S - 1] : 0;
  if ((rc = ensure(g, g->b_fold, (size_t)16 * W))) return rc;
  if ((rc = waypoint_sets_impl(g, af, ptr<int32_t>(g->b_reach), nullptr, 1, W, 0, fp->eps2, fp->eps2_max,
                               nullptr, &ga, fold ? ptr<int32_t>(g->b_fold) : nullptr)))
    return rc;
  if ((rc = ensure(g, g->b_tposes, tpose_bytes * W))) return rc;
  if ((rc = ensure(g, g->b_poses, pose_bytes * W))) return rc;
  if ((rc = ensure(g, g->b_relax, (size_t)8 * W))) return rc;
  if ((rc = ensure(g, g->b_status, 4))) return rc;
  int32_t* tposes = ptr<int32_t>(g->b_tposes);
  // the last waypoint's follower pose: the reach pose's joints 0 .. F
  CK(cudaMemcpyAsync(tposes + (long)(W - 1) * 3 * (F + 1), g->b_reach.p, tpose_bytes,
                     cudaMemcpyDeviceToDevice, g->st));
  ik_path_params pp{W, 0, fp->eps2, fp->eps2_max, fp->max_relax};
  if ((rc = chain_impl(g, af, &pp, 1, 0, 0, nullptr, tposes, ptr<int32_t>(g->b_relax),
                       ptr<int32_t>(g->b_status), nullptr, rad)))
    return rc;
  int32_t* dposes = fold ? ptr<int32_t>(g->b_poses) : tposes;
  if (fold) {
    ProfScope ps(g, P_CHAIN);
    CK(launch_fold_last(g->d, ad.seg[S - 1], S, 1, W, tposes, ptr<int32_t>(g->b_fold), dposes,
                        ptr<int32_t>(g->b_relax), ptr<int32_t>(g->b_status), g->st));
  }
  int32_t st = 0;
  if ((rc = copy_out(g, poses_out, dposes, pose_bytes * W, 0))) return rc;
  if ((rc = copy_out(g, relax_out, g->b_relax.p, (size_t)8 * W, 0))) return rc;
  if ((rc = copy_out(g, &st, g->b_status.p, 4, 0))) return rc;
  if ((rc = sync(g))) return rc;
  *status = st;
  return IK_OK;
}

int ik_plan_path_short(ik_grid g, const ik_arm* arm, const int32_t* reach_pose, const ik_path_params* pp,
                       int k_max, int32_t* poses_out, int32_t* relax_out, int* status, int32_t* shortcut_out,
                       int32_t* guide_pose_out) {
  int rc = set_device(g);
  if (rc) return rc;
  if (!reach_pose || !poses_out || !relax_out || !status || !shortcut_out) return IK_ERR_ARG;
  if ((rc = check_path_params(pp))) return rc;
  if ((rc = check_arm(arm))) return rc;
  const int S = arm->n_seg, W = pp->n_way;
  if (k_max < 1 || k_max > S) return IK_ERR_ARG;
  if (arm_limits(g, arm)) return IK_ERR_UNSUPPORTED;
  ArmDev ad;
  std::vector<std::pair<int, int>> key;
  if ((rc = resolve_arm(g, arm, reach_pose, &ad, &key))) return rc;
  const size_t pose_bytes = (size_t)12 * (S + 1);
  shortcut_out[0] = shortcut_out[1] = 0;
  // the reach pose must be a valid pose of this arm in this grid
  if ((rc = to_device(g, g->b_reach, reach_pose, pose_bytes))) return rc;
  if ((rc = ensure(g, g->b_valid, 4))) return rc;
  if ((rc = validate_impl(g, ad, ptr<int32_t>(g->b_reach), 1, ptr<int32_t>(g->b_valid)))) return rc;
  int32_t valid = 0;
  if ((rc = copy_out(g, &valid, g->b_valid.p, 4, 0))) return rc;
  if ((rc = sync(g))) return rc;
  if (!valid) {
    *status = IK_PATH_UNREACHABLE;
    return IK_OK;
  }
  // the shortcut: the first virtual arm L_1 .. L_{k-1}, l (k = 1 .. k_max, then
  // l = 1 .. L_k) whose reach search from the root finds the target
  const int32_t* root = reach_pose;
  const int32_t* target = reach_pose + 3 * S;
  GuideArm ga;
  ga.S = S;
  for (int k = 0; k < S; ++k) ga.len[k] = arm->len[k];
  std::vector<int32_t> gpose(reach_pose, reach_pose + 3 * (S + 1));
  bool found = false;
  for (int k = 1; k <= k_max && !found; ++k) {
    for (int l = 1; l <= arm->len[k - 1] && !found; ++l) {
      int32_t vlen[IK_MAX_SEG];
      for (int q = 0; q < k; ++q) vlen[q] = arm->len[q];
      vlen[k - 1] = l;
      const ik_arm va{k, vlen, arm->tol};
      ArmDev av;
      std::vector<std::pair<int, int>> keyv;
      if ((rc = resolve_arm(g, &va, root, &av, &keyv))) return rc;
      int32_t *d_vpose = nullptr, *d_vfound = nullptr;
      if ((rc = reach_many_impl(g, av, keyv, root, target, 1, nullptr, nullptr, nullptr, 0, &d_vpose,
                                &d_vfound)))
        return rc;
      int32_t vfound = 0;
      std::vector<int32_t> vpose((size_t)3 * (k + 1));
      if ((rc = copy_out(g, &vfound, d_vfound, 4, 0))) return rc;
      if ((rc = copy_out(g, vpose.data(), d_vpose, (size_t)12 * (k + 1), 0))) return rc;
      if ((rc = sync(g))) return rc;
      if (vfound) {
        found = true;
        shortcut_out[0] = k;
        shortcut_out[1] = l;
        ga.S = k;
        for (int q = 0; q < k; ++q) ga.len[q] = vlen[q];
        gpose = vpose;
      }
    }
  }
  if (found && guide_pose_out) memcpy(guide_pose_out, gpose.data(), gpose.size() * 4);
  // the guide pose in a buffer that the actual arm's steps do not use; the
  // actual arm's tables are resolved again (the virtual arms may share its
  // shells, whose edge-mask boxes can have grown)
  if ((rc = to_device(g, g->b_targets, gpose.data(), gpose.size() * 4))) return rc;
  if ((rc = resolve_arm(g, arm, reach_pose, &ad, &key))) return rc;
  if ((rc = ensure_forward(g, ad, key, reach_pose))) return rc;
  if ((rc = to_device(g, g->b_reach, reach_pose, pose_bytes))) return rc;
  if ((rc = waypoint_sets_impl(g, ad, ptr<int32_t>(g->b_targets), nullptr, 1, W, 0, pp->eps2, pp->eps2_max,
                               nullptr, &ga)))
    return rc;
  if ((rc = ensure(g, g->b_poses, pose_bytes * W))) return rc;
  if ((rc = ensure(g, g->b_relax, (size_t)8 * W))) return rc;
  if ((rc = ensure(g, g->b_status, 4))) return rc;
  int32_t* dposes = ptr<int32_t>(g->b_poses);
  CK(cudaMemcpyAsync(dposes + (long)(W - 1) * 3 * (S + 1), g->b_reach.p, pose_bytes,
                     cudaMemcpyDeviceToDevice, g->st));
  if ((rc = chain_impl(g, ad, pp, 1, 0, 0, nullptr, dposes, ptr<int32_t>(g->b_relax),
                       ptr<int32_t>(g->b_status))))
    return rc;
  int32_t st = 0;
  if ((rc = copy_out(g, poses_out, dposes, pose_bytes * W, 0))) return rc;
  if ((rc = copy_out(g, relax_out, g->b_relax.p, (size_t)8 * W, 0))) return rc;
  if ((rc = copy_out(g, &st, g->b_status.p, 4, 0))) return rc;
  if ((rc = sync(g))) return rc;
  *status = st;
  return IK_OK;
}

int ik_plan_between(ik_grid g, const ik_arm* arm, const int32_t* start_pose, const ik_arm* guide_arm,
                    const int32_t target[3], const ik_path_params* pp, int32_t* poses_out,
                    int32_t* relax_out, int32_t* guide_pose_out, int* status) {
  int rc = set_device(g);
  if (rc) return rc;
  if (!start_pose || !target || !poses_out || !relax_out || !status) return IK_ERR_ARG;
  if ((rc = check_path_params(pp))) return rc;
  if ((rc = check_arm(guide_arm))) return rc;
  ArmDev ad, av;
  std::vector<std::pair<int, int>> key, keyv;
  if ((rc = resolve_arm(g, arm, start_pose, &ad, &key))) return rc;
  const int S = ad.S, Sv = guide_arm->n_seg, W = pp->n_way;
  const size_t pose_bytes = (size_t)12 * (S + 1);
  for (int k = 0; k <= S; ++k)
    if (!point_inside(g->d, start_pose + 3 * k)) return IK_ERR_ARG;
  if (!point_inside(g->d, target)) return IK_ERR_ARG;
  auto unreachable = [&]() {
    for (int j = 0; j < W; ++j) {
      memcpy(poses_out + (size_t)j * 3 * (S + 1), start_pose, pose_bytes);
      relax_out[2 * j] = j == 0 ? 0 : -1;
      relax_out[2 * j + 1] = 0;
    }
    *status = IK_PATH_UNREACHABLE;
    return sync(g);
  };
  // the start must be a valid pose of this arm in this grid
  if ((rc = to_device(g, g->b_old, start_pose, pose_bytes))) return rc;
  if ((rc = ensure(g, g->b_valid, 4))) return rc;
  if ((rc = validate_impl(g, ad, ptr<int32_t>(g->b_old), 1, ptr<int32_t>(g->b_valid)))) return rc;
  int32_t valid = 0;
  if ((rc = copy_out(g, &valid, g->b_valid.p, 4, 0))) return rc;
  if ((rc = sync(g))) return rc;
  if (!valid) return unreachable();
  // the virtual arm reaches from the start's end effector for the target
  const int32_t* vroot = start_pose + 3 * S;
  if ((rc = resolve_arm(g, guide_arm, vroot, &av, &keyv))) return rc;
  int32_t *d_vpose = nullptr, *d_vfound = nullptr;
  if ((rc = reach_many_impl(g, av, keyv, vroot, target, 1, nullptr, nullptr, nullptr, 0, &d_vpose,
                            &d_vfound)))
    return rc;
  int32_t vfound = 0;
  std::vector<int32_t> vpose((size_t)3 * (Sv + 1));
  if ((rc = copy_out(g, &vfound, d_vfound, 4, 0))) return rc;
  if ((rc = copy_out(g, vpose.data(), d_vpose, (size_t)12 * (Sv + 1), 0))) return rc;
  if ((rc = sync(g))) return rc;
  if (!vfound) return unreachable();
  if (guide_pose_out) memcpy(guide_pose_out, vpose.data(), (size_t)12 * (Sv + 1));
  // the guide pose in a buffer that the actual arm's steps do not use
  if ((rc = to_device(g, g->b_targets, vpose.data(), (size_t)12 * (Sv + 1)))) return rc;
  const int32_t* d_guide = ptr<int32_t>(g->b_targets);
  // the actual arm: forward sets from its root, waypoint sets j >= 1 along the
  // guide, the forward chain from the start pose.  Its tables are resolved
  // again: the virtual arm's shells may be the same tables, whose edge-mask
  // boxes (and buffers) grew for the virtual root.
  if ((rc = resolve_arm(g, arm, start_pose, &ad, &key))) return rc;
  if ((rc = ensure_forward(g, ad, key, start_pose))) return rc;
  GuideArm ga;
  ga.S = Sv;
  for (int k = 0; k < Sv; ++k) ga.len[k] = guide_arm->len[k];
  if ((rc = ensure(g, g->b_found, 4))) return rc;
  CK(cudaMemcpyAsync(ptr<int32_t>(g->b_found), &vfound, 4, cudaMemcpyHostToDevice, g->st));
  if ((rc = waypoint_sets_impl(g, ad, d_guide, ptr<int32_t>(g->b_found), 1, W, 1, pp->eps2, pp->eps2_max,
                               nullptr, &ga)))
    return rc;
  if ((rc = ensure(g, g->b_poses, pose_bytes * W))) return rc;
  if ((rc = ensure(g, g->b_relax, (size_t)8 * W))) return rc;
  if ((rc = ensure(g, g->b_status, 4))) return rc;
  int32_t* dposes = ptr<int32_t>(g->b_poses);
  CK(cudaMemcpyAsync(dposes, start_pose, pose_bytes, cudaMemcpyHostToDevice, g->st));
  if ((rc = chain_impl(g, ad, pp, 1, 1, 0, ptr<int32_t>(g->b_found), dposes, ptr<int32_t>(g->b_relax),
                       ptr<int32_t>(g->b_status))))
    return rc;
  if ((rc = copy_out(g, poses_out, dposes, pose_bytes * W, 0))) return rc;
  if ((rc = copy_out(g, relax_out, g->b_relax.p, (size_t)8 * W, 0))) return rc;
  if ((rc = copy_out(g, status, g->b_status.p, 4, 0))) return rc;
  return sync(g);
}

int ik_reach_path_many(ik_grid g, const ik_arm* arm, const int32_t root[3], const int32_t* targets,
                       int n, const ik_path_params* pp, int32_t* reach_out, int32_t* found_out,
                       int32_t* poses_out, int32_t* relax_out, int32_t* status_out, int on_device) {
  int rc = set_device(g);
  if (rc) return rc;
  if (!root || !point_inside(g->d, root) || n < 0 || (n > 0 && !targets)) return IK_ERR_ARG;
  if ((rc = check_path_params(pp))) return rc;
  if (n == 0) return IK_OK;
  if (!on_device)
    for (int i = 0; i < n; ++i)
      if (!point_inside(g->d, targets + 3 * i)) return IK_ERR_ARG;
  ArmDev ad;
  std::vector<std::pair<int, int>> key;
  if ((rc = resolve_arm(g, arm, root, &ad, &key))) return rc;
  const int S = ad.S, W = pp->n_way;
  const size_t pose_bytes = (size_t)12 * (S + 1);
  int32_t *d_reach = nullptr, *d_found = nullptr;
  if ((rc = reach_many_impl(g, ad, key, root, targets, n, on_device ? reach_out : nullptr,
                            on_device ? found_out : nullptr, nullptr, on_device, &d_reach, &d_found)))
    return rc;
  if ((rc = waypoint_sets_impl(g, ad, d_reach, d_found, n, W, 0, pp->eps2, pp->eps2_max))) return rc;
  int32_t *dposes = poses_out, *drelax = relax_out, *dstatus = status_out;
  if (!on_device) {
    if ((rc = ensure(g, g->b_poses, pose_bytes * W * n))) return rc;
    if ((rc = ensure(g, g->b_relax, (size_t)8 * W * n))) return rc;
    if ((rc = ensure(g, g->b_status, (size_t)4 * n))) return rc;
    dposes = ptr<int32_t>(g->b_poses);
    drelax = ptr<int32_t>(g->b_relax);
    dstatus = ptr<int32_t>(g->b_status);
  }
  // pose W-1 of each path is its reach pose
  CK(cudaMemcpy2DAsync(dposes + (long)(W - 1) * 3 * (S + 1), pose_bytes * W, d_reach, pose_bytes,
                       pose_bytes, n, cudaMemcpyDeviceToDevice, g->st));
  if ((rc = chain_impl(g, ad, pp, n, 0, 0, d_found, dposes, drelax, dstatus))) return rc;
  if (!on_device) {
    if ((rc = copy_out(g, reach_out, d_reach, pose_bytes * n, 0))) return rc;
    if ((rc = copy_out(g, found_out, d_found, (size_t)4 * n, 0))) return rc;
    if ((rc = copy_out(g, poses_out, dposes, pose_bytes * W * n, 0))) return rc;
    if ((rc = copy_out(g, relax_out, drelax, (size_t)8 * W * n, 0))) return rc;
    if ((rc = copy_out(g, status_out, dstatus, (size_t)4 * n, 0))) return rc;
  }
  return sync(g);
}

// The whole reach + path pipeline for n slots, enqueued on the grid's stream
// with no host transfer, allocation or synchronisation (every buffer was
// sized by a warm-up call): rasterise the boxes, rebuild every edge mask and
// the forward sets, then reach, waypoint sets and smooth chains.
static int enqueue_reach_path(ik_grid g, const ArmDev& ad, const std::vector<ShellDev*>& used,
                              const int32_t* d_root, const int32_t* d_boxes, int n_boxes,
                              const int32_t* d_targets, int n,
                              const ik_path_params* pp, int32_t* d_reach, int32_t* d_found,
                              int32_t* d_poses, int32_t* d_relax, int32_t* d_status) {
  const Dims& d = g->d;
  const int S = ad.S, W = pp->n_way;
  const long qs = (long)(S + 1) * d.nw;
  const size_t pose_bytes = (size_t)12 * (S + 1);
  int rc;
  CK(launch_rasterize(d, d_boxes, n_boxes, g->d_occ_raw, g->st));
  if ((rc = apply_dilation(g))) return rc;
  if (g->use_masks)
    for (ShellDev* sh : used) CK(launch_masks(g, *sh, sh->mbox, sh->d_mask));
  uint32_t* F = ptr<uint32_t>(g->F);
  int32_t* fb = ptr<int32_t>(g->F_box);
  CK(cudaMemsetAsync(fb, kBoxEmptyByte, (size_t)(S + 1) * 24, g->st));
  CK(launch_seed_points(d, d_root, 1, nullptr, g->d_occ, F, d.nw, nullptr, fb, 0, g->st));
  for (int k = 1; k <= S; ++k)
    CK(launch_propagate(d, g->tc, ad.segf[k - 1], F + (k - 1) * d.nw, 0, nullptr, 0, g->d_occ,
                        F + k * d.nw, 0, 1, fb + 6 * (k - 1), fb + 6 * k, 0, g->st));
  uint32_t* V = ptr<uint32_t>(g->V);
  int32_t* vb = ptr<int32_t>(g->V_box);
  CK(cudaMemsetAsync(vb, kBoxEmptyByte, (size_t)n * (S + 1) * 24, g->st));
  CK(launch_seed_points(d, d_targets, n, F + (long)S * d.nw, nullptr, V + (long)S * d.nw, qs, nullptr,
                        vb + 6 * S, 6L * (S + 1), g->st));
  if ((rc = backward_sets(g, ad, V, n, P_BWD_REACH, vb))) return rc;
  CK(launch_traceback(d, ad, d_root, V, qs, n, d_reach, d_found, g->st));
  if ((rc = waypoint_sets_impl(g, ad, d_reach, d_found, n, W, 0, pp->eps2, pp->eps2_max))) return rc;
  CK(cudaMemcpy2DAsync(d_poses + (long)(W - 1) * 3 * (S + 1), pose_bytes * W, d_reach, pose_bytes,
                       pose_bytes, n, cudaMemcpyDeviceToDevice, g->st));
  return chain_impl(g, ad, pp, n, 0, 0, d_found, d_poses, d_relax, d_status);
}

int ik_batch_capture(ik_grid g, const ik_arm* arm, const int32_t root[3], const int32_t* boxes_dev,
                     int n_boxes, const int32_t* targets_dev, int n, const ik_path_params* pp,
                     int32_t* reach_dev, int32_t* found_dev, int32_t* poses_dev, int32_t* relax_dev,
                     int32_t* status_dev, ik_batch* out) {
  int rc = set_device(g);
  if (rc) return rc;
  if (!out || !root || !point_inside(g->d, root) || n < 1 || !targets_dev || n_boxes < 0 ||
      (n_boxes > 0 && !boxes_dev) || !reach_dev || !found_dev || !poses_dev || !relax_dev ||
      !status_dev)
    return IK_ERR_ARG;
  if ((rc = check_path_params(pp))) return rc;
  if (!g->st) return IK_ERR_STATE;  // the legacy default stream cannot be captured
  *out = nullptr;
  ArmDev ad;
  std::vector<std::pair<int, int>> key;
  std::vector<ShellDev*> used;
  // warm-up: size every buffer and build every table with one ordinary run
  if ((rc = ik_set_boxes(g, boxes_dev, n_boxes, 1))) return rc;
  if ((rc = ik_reach_path_many(g, arm, root, targets_dev, n, pp, reach_dev, found_dev, poses_dev,
                               relax_dev, status_dev, 1)))
    return rc;
  if ((rc = resolve_arm(g, arm, root, &ad, &key, &used))) return rc;
  // the root is the batch's own input: ordinary calls reuse the grid's buffer
  int32_t* d_root = nullptr;
  CK(cudaMalloc(&d_root, 16));
  if (cudaMemcpy(d_root, root, 12, cudaMemcpyHostToDevice) != cudaSuccess || (rc = sync(g))) {
    cudaFree(d_root);
    return rc ? rc : IK_ERR_CUDA;
  }
  const bool prof = g->prof_on, cnt = g->count_on;
  g->prof_on = g->count_on = false;
  g->capturing = true;
  cudaError_t e = cudaStreamBeginCapture(g->st, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    rc = enqueue_reach_path(g, ad, used, d_root, boxes_dev, n_boxes, targets_dev, n, pp, reach_dev,
                            found_dev, poses_dev, relax_dev, status_dev);
  } else {
    rc = fail_cuda(e);
  }
  cudaGraph_t graph = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(g->st, &graph);
  g->capturing = false;
  g->prof_on = prof;
  g->count_on = cnt;
  forget_device_state(g);
  if (rc || e2 != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    cudaFree(d_root);
    return rc ? rc : fail_cuda(e2);
  }
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, graph, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(graph);
    cudaFree(d_root);
    return fail_cuda(e);
  }
  ik_batch b = new ik_batch_s();
  b->g = g;
  b->graph = graph;
  b->exec = exec;
  memcpy(b->root, root, 12);
  b->d_root = d_root;
  b->key = key;
  b->used = used;
  b->gen = g->buf_gen;
  ++g->live_batches;
  *out = b;
  return IK_OK;
}

int ik_batch_launch(ik_batch b) {
  if (!b) return IK_ERR_ARG;
  ik_grid g = b->g;
  int rc = set_device(g);
  if (rc) return rc;
  CK(cudaGraphLaunch(b->exec, g->st));
  // the replay leaves a new occupancy with its edge masks and forward sets:
  // later calls on this stream may use them as they are, unless the grid
  // has replaced a buffer (or a mask layout) since the capture, in which
  // case the replay wrote buffers of its own
  forget_device_state(g);
  if (b->gen != g->buf_gen) return IK_OK;
  if (g->use_masks)
    for (ShellDev* sh : b->used) sh->mask_version = g->version;
  g->f_valid = true;
  g->f_version = g->version;
  g->f_key = b->key;
  memcpy(g->f_root, b->root, 12);
  return IK_OK;
}

int ik_batch_destroy(ik_batch b) {
  if (!b) return IK_ERR_ARG;
  cudaSetDevice(b->g->device);
  cudaStreamSynchronize(b->g->st);
  cudaGraphExecDestroy(b->exec);
  cudaGraphDestroy(b->graph);
  cudaFree(b->d_root);
  ik_grid g = b->g;
  if (--g->live_batches == 0) {
    for (void* p : g->retired) cudaFree(p);
    g->retired.clear();
  }
  delete b;
  return IK_OK;
}

int ik_replan(ik_grid g, const ik_arm* arm, const int32_t* poses_in, int n_way, int current_idx,
              const ik_path_params* pp, int32_t* poses_out, int32_t* relax_out, int* status) {
  int rc = set_device(g);
  if (rc) return rc;
  if (!poses_in || !poses_out || !relax_out || !status || n_way < 2 || current_idx < 0 ||
      current_idx >= n_way)
    return IK_ERR_ARG;
  if ((rc = check_path_params(pp))) return rc;
  if (pp->n_way != n_way) return IK_ERR_ARG;
  ArmDev ad;
  std::vector<std::pair<int, int>> key;
  if ((rc = resolve_arm(g, arm, poses_in, &ad, &key))) return rc;
  const int S = ad.S, W = n_way, c = current_idx;
  const size_t pose_bytes = (size_t)12 * (S + 1);
  const int32_t* root = poses_in;
  for (int j = 0; j < W; ++j)
    if (poses_in[3 * (S + 1) * j] != root[0] || poses_in[3 * (S + 1) * j + 1] != root[1] ||
        poses_in[3 * (S + 1) * j + 2] != root[2])
      return IK_ERR_ARG;
  if (!point_inside(g->d, root)) return IK_ERR_ARG;
  // 1. is the remainder still valid?
  if ((rc = ensure(g, g->b_poses, pose_bytes * W))) return rc;
  int32_t* dposes = ptr<int32_t>(g->b_poses);
  CK(cudaMemcpyAsync(dposes, poses_in, pose_bytes * W, cudaMemcpyHostToDevice, g->st));
  if ((rc = ensure(g, g->b_valid, (size_t)4 * W))) return rc;
  if ((rc = validate_impl(g, ad, dposes, W, ptr<int32_t>(g->b_valid)))) return rc;
  std::vector<int32_t> valid(W);
  if ((rc = copy_out(g, valid.data(), g->b_valid.p, (size_t)4 * W, 0))) return rc;
  if ((rc = sync(g))) return rc;
  bool cut = false;
  for (int j = c + 1; j < W; ++j)
    if (!valid[j]) cut = true;
  for (int j = 0; j < 2 * W; ++j) relax_out[j] = 0;
  if (!cut) {
    memcpy(poses_out, poses_in, pose_bytes * W);
    *status = IK_PATH_KEPT;
    return IK_OK;
  }
  // 2. forward sets on the new occupancy; 3. the guiding reach pose
  if ((rc = ensure_forward(g, ad, key, root))) return rc;
  if ((rc = ensure(g, g->b_reach, pose_bytes))) return rc;
  int32_t* dreach = ptr<int32_t>(g->b_reach);
  const int32_t* old_reach = poses_in + (size_t)3 * (S + 1) * (W - 1);
  if (valid[W - 1]) {
    CK(cudaMemcpyAsync(dreach, old_reach, pose_bytes, cudaMemcpyHostToDevice, g->st));
  } else {
    const long qs = (long)(S + 1) * g->d.nw;
    if ((rc = ensure(g, g->V, (size_t)qs * 4))) return rc;
    if ((rc = to_device(g, g->b_targets, old_reach + 3 * S, 12))) return rc;
    if ((rc = to_device(g, g->b_old, old_reach, pose_bytes))) return rc;
    if ((rc = to_device(g, g->b_root, root, 12))) return rc;
    if ((rc = ensure(g, g->b_found, 4))) return rc;
    uint32_t* V = ptr<uint32_t>(g->V);
    const uint32_t* F = ptr<uint32_t>(g->F);
    if ((rc = ensure(g, g->V_box, (size_t)(S + 1) * 24))) return rc;
    int32_t* vb = ptr<int32_t>(g->V_box);
    CK(cudaMemsetAsync(vb, kBoxEmptyByte, (size_t)(S + 1) * 24, g->st));
    CK(launch_seed_points(g->d, ptr<int32_t>(g->b_targets), 1, F + (long)S * g->d.nw, nullptr,
                          V + (long)S * g->d.nw, qs, nullptr, vb + 6 * S, 0, g->st));
    if ((rc = backward_sets(g, ad, V, 1, P_BWD_REACH, vb))) return rc;
    CK(launch_traceback_nearest(g->d, ad, ptr<int32_t>(g->b_root), V, ptr<int32_t>(g->b_old), dreach,
                                ptr<int32_t>(g->b_found), g->st));
    int32_t found = 0;
    if ((rc = copy_out(g, &found, g->b_found.p, 4, 0))) return rc;
    if ((rc = sync(g))) return rc;
    if (!found) {
      memcpy(poses_out, poses_in, pose_bytes * (c + 1));
      for (int j = c + 1; j < W; ++j) {
        memcpy(poses_out + (size_t)3 * (S + 1) * j, poses_in + (size_t)3 * (S + 1) * c, pose_bytes);
        relax_out[2 * j] = -1;
      }
      *status = IK_PATH_UNREACHABLE;
      return IK_OK;
    }
  }
  // 4. guide + survivor sets of waypoints c+1 .. W-1; 5. forward chain
  if ((rc = waypoint_sets_impl(g, ad, dreach, nullptr, 1, W, c + 1, pp->eps2, pp->eps2_max))) return rc;
  if ((rc = ensure(g, g->b_relax, (size_t)8 * W))) return rc;
  if ((rc = ensure(g, g->b_status, 4))) return rc;
  if ((rc = chain_impl(g, ad, pp, 1, 1, c, nullptr, dposes, ptr<int32_t>(g->b_relax),
                       ptr<int32_t>(g->b_status))))
    return rc;
  int32_t st = 0;
  if ((rc = copy_out(g, poses_out, dposes, pose_bytes * W, 0))) return rc;
  if ((rc = copy_out(g, relax_out, g->b_relax.p, (size_t)8 * W, 0))) return rc;
  if ((rc = copy_out(g, &st, g->b_status.p, 4, 0))) return rc;
  if ((rc = sync(g))) return rc;
  *status = st;
  return IK_OK;
}

// Batched replan for R slots, enqueued with no host synchronisation:
// validate every pose, decide per slot (live, cut, reach pose to re-solve),
// re-solve the cut reach poses, then survivor sets of the waypoints after
// each slot's current index and the forward smooth chains.  All pointers are
// device pointers; the forward sets of `root` must be current (g->F, b_root).
static int enqueue_replan(ik_grid g, const ArmDev& ad, const int32_t* d_poses_in, const int32_t* d_c,
                          int R, const ik_path_params* pp, int32_t* d_poses_out, int32_t* d_relax,
                          int32_t* d_status) {
  const Dims& d = g->d;
  const int S = ad.S, W = pp->n_way;
  const long ps = 3L * (S + 1), qs = (long)(S + 1) * d.nw;
  int rc;
  if ((rc = ensure(g, g->b_rp, (size_t)4 * ((size_t)R * W + 3 * R + 3 * R + R * ps + 2 * R)))) return rc;
  if ((rc = ensure(g, g->V, (size_t)R * qs * 4))) return rc;
  if ((rc = ensure(g, g->V_box, (size_t)R * (S + 1) * 24))) return rc;
  int32_t* valid = ptr<int32_t>(g->b_rp);
  int32_t* cut = valid + (long)R * W;
  int32_t* need = cut + R;
  int32_t* gate = need + R;
  int32_t* tgt = gate + R;
  int32_t* reach = tgt + 3L * R;
  int32_t* rfound = reach + (long)R * ps;
  uint32_t* V = ptr<uint32_t>(g->V);
  int32_t* vb = ptr<int32_t>(g->V_box);
  const uint32_t* F = ptr<uint32_t>(g->F);
  CK(cudaMemcpyAsync(d_poses_out, d_poses_in, (size_t)R * W * ps * 4, cudaMemcpyDeviceToDevice, g->st));
  CK(cudaMemsetAsync(d_status, 0xff, (size_t)R * 4, g->st));
  CK(cudaMemsetAsync(rfound, 0, (size_t)R * 4, g->st));
  {
    ProfScope ps_(g, P_VALIDATE);
    CK(launch_validate(d, ad, g->d_occ, d_poses_in, R * W, valid, g->st));
  }
  CK(launch_replan_prepare(R, W, S, d_poses_in, d_c, valid, cut, need, tgt, d_relax, g->st));
  CK(cudaMemsetAsync(vb, kBoxEmptyByte, (size_t)R * (S + 1) * 24, g->st));
  CK(launch_seed_points(d, tgt, R, F + (long)S * d.nw, nullptr, V + (long)S * d.nw, qs, need,
                        vb + 6 * S, 6L * (S + 1), g->st));
  if ((rc = backward_sets(g, ad, V, R, P_BWD_REACH, vb))) return rc;
  CK(launch_traceback_nearest_many(d, ad, ptr<int32_t>(g->b_root), V, qs, d_poses_in + (long)(W - 1) * ps,
                                   (long)W * ps, reach, rfound, need, R, g->st));
  CK(launch_replan_fix(R, W, S, d_poses_in, cut, need, reach, rfound, gate, g->st));
  if ((rc = waypoint_sets_impl(g, ad, reach, gate, R, W, 0, pp->eps2, pp->eps2_max, d_c))) return rc;
  if ((rc = chain_impl(g, ad, pp, R, 1, 0, gate, d_poses_out, d_relax, d_status, d_c))) return rc;
  CK(launch_replan_finalize(R, W, S, d_c, cut, gate, d_poses_out, d_relax, d_status, g->st));
  return IK_OK;
}

int ik_replan_many(ik_grid g, const ik_arm* arm, const int32_t root[3], const int32_t* poses_in,
                   const int32_t* current, int n, const ik_path_params* pp, int32_t* poses_out,
                   int32_t* relax_out, int32_t* status_out, int on_device) {
  int rc = set_device(g);
  if (rc) return rc;
  if (!root || !point_inside(g->d, root) || n < 0 ||
      (n > 0 && (!poses_in || !current || !poses_out || !relax_out || !status_out)))
    return IK_ERR_ARG;
  if ((rc = check_path_params(pp))) return rc;
  if (n == 0) return IK_OK;
  ArmDev ad;
  std::vector<std::pair<int, int>> key;
  if ((rc = resolve_arm(g, arm, root, &ad, &key))) return rc;
  const int S = ad.S, W = pp->n_way;
  const size_t path_bytes = (size_t)12 * (S + 1) * W;
  if (!on_device) {
    for (int r = 0; r < n; ++r) {
      if (current[r] < 0 || current[r] >= W) continue;
      const int32_t* P = poses_in + (size_t)3 * (S + 1) * W * r;
      for (int j = 0; j < W; ++j)
        if (P[3 * (S + 1) * j] != root[0] || P[3 * (S + 1) * j + 1] != root[1] ||
            P[3 * (S + 1) * j + 2] != root[2])
          return IK_ERR_ARG;
    }
  }
  if ((rc = ensure_forward(g, ad, key, root))) return rc;
  if ((rc = to_device(g, g->b_root, root, 12))) return rc;
  const int32_t *dpin = poses_in, *dc = current;
  int32_t *dpout = poses_out, *drelax = relax_out, *dstatus = status_out;
  if (!on_device) {
    if ((rc = to_device(g, g->b_rin, poses_in, path_bytes * n))) return rc;
    if ((rc = to_device(g, g->b_rc, current, (size_t)4 * n))) return rc;
    if ((rc = ensure(g, g->b_poses, path_bytes * n))) return rc;
    if ((rc = ensure(g, g->b_relax, (size_t)8 * W * n))) return rc;
    if ((rc = ensure(g, g->b_status, (size_t)4 * n))) return rc;
    dpin = ptr<int32_t>(g->b_rin);
    dc = ptr<int32_t>(g->b_rc);
    dpout = ptr<int32_t>(g->b_poses);
    drelax = ptr<int32_t>(g->b_relax);
    dstatus = ptr<int32_t>(g->b_status);
  }
  if ((rc = enqueue_replan(g, ad, dpin, dc, n, pp, dpout, drelax, dstatus))) return rc;
  if (!on_device) {
    if ((rc = copy_out(g, poses_out, dpout, path_bytes * n, 0))) return rc;
    if ((rc = copy_out(g, relax_out, drelax, (size_t)8 * W * n, 0))) return rc;
    if ((rc = copy_out(g, status_out, dstatus, (size_t)4 * n, 0))) return rc;
  }
  return sync(g);
}

int ik_set_option(ik_grid g, int option, int value) {
  int rc = set_device(g);
  if (rc) return rc;
  if (option == IK_OPT_TILE_DEPTH) {
    if (value != 8 && value != 16) return IK_ERR_ARG;
    g->tc.depth = value;
    return IK_OK;
  }
  if (option == IK_OPT_QUERY_PAIRS) {
    if (value < 0 || value > 2) return IK_ERR_ARG;
    g->tc.pair = value;
    return IK_OK;
  }
  if (option == IK_OPT_ROW_LANES) {
    if (value != 0 && value != 1) return IK_ERR_ARG;
    g->tc.rows = value;
    return IK_OK;
  }
  if (option == IK_OPT_TMA_MASKS) {
    if (value != 0 && value != 1) return IK_ERR_ARG;
    g->use_tma = value;
    return IK_OK;
  }
  if (option == IK_OPT_WORK_LIST) {
    if (value < 0 || value > 2) return IK_ERR_ARG;
    g->work_list = value;
    return IK_OK;
  }
  if (option == IK_OPT_DILATE_R2) {
    if (value < 0 || value > 100) return IK_ERR_ARG;
    g->dilate_r2 = value;
    if ((rc = apply_dilation(g))) return rc;
    ++g->version;
    return sync(g);
  }
  if (option != IK_OPT_EDGE_MASKS) return IK_ERR_ARG;
  if ((rc = sync(g))) return rc;
  g->use_masks = value != 0;
  if (!g->use_masks) {
    std::vector<ShellDev*> all;
    for (auto& kv : g->shells) all.push_back(kv.second);
    for (auto& kv : g->cone_shells) all.push_back(kv.second);
    for (ShellDev* sh : all) {
      if ((rc = release(g, sh->d_mask))) return rc;
      sh->d_mask = nullptr;
      sh->mask_bytes = 0;
      sh->mbox = MaskBox{0, 0, 0, -1, -1, -1};
      sh->mask_version = ~0ull;
    }
  }
  return IK_OK;
}

int ik_profile_enable(ik_grid g, int timing, int counting) {
  int rc = set_device(g);
  if (rc) return rc;
  if (counting && !g->d_counters) {
    CK(cudaMalloc(&g->d_counters, sizeof(unsigned long long) * kCounters * P_N));
    CK(cudaMemsetAsync(g->d_counters, 0, sizeof(unsigned long long) * kCounters * P_N, g->st));
  }
  g->prof_on = timing != 0;
  g->count_on = counting != 0;
  g->h_counters.assign(kCounters * P_N, 0ull);
  return sync(g);
}

int ik_profile_read(ik_grid g, double* ms_out, int64_t* launches_out, uint64_t* counters_out,
                    int cap) {
  int rc = set_device(g);
  if (rc) return rc;
  if ((rc = sync(g))) return rc;
  std::vector<double> ms(P_N, 0.0);
  std::vector<int64_t> n(P_N, 0);
  for (auto& r : g->recs) {
    float t = 0.f;
    CK(cudaEventElapsedTime(&t, r.a, r.b));
    ms[r.id] += t;
    n[r.id] += 1;
  }
  g->recs.clear();
  g->ev_used = 0;
  std::vector<unsigned long long> cnt(kCounters * P_N, 0);
  if (g->d_counters) {
    CK(cudaMemcpy(cnt.data(), g->d_counters, sizeof(unsigned long long) * kCounters * P_N,
                  cudaMemcpyDeviceToHost));
    CK(cudaMemset(g->d_counters, 0, sizeof(unsigned long long) * kCounters * P_N));
  }
  if (g->h_counters.size() == cnt.size())
    for (size_t i = 0; i < cnt.size(); ++i) {
      cnt[i] += g->h_counters[i];
      g->h_counters[i] = 0;
    }
  for (int i = 0; i < P_N && i < cap; ++i) {
    if (ms_out) ms_out[i] = ms[i];
    if (launches_out) launches_out[i] = n[i];
    if (counters_out)
      for (int j = 0; j < kCounters; ++j) counters_out[kCounters * i + j] = cnt[kCounters * i + j];
  }
  return P_N;
}

const char* ik_profile_name(int i) { return (i >= 0 && i < P_N) ? kProfNames[i] : ""; }

int ik_shell_offsets(int len, float tol, int32_t* lo2_hi2, int32_t* offs_out, int cap) {
  if (len < 1 || len > IK_MAX_LEN || !(tol >= 0.0f && tol < 1.0f)) return IK_ERR_ARG;
  int lo2, hi2;
  shell_bounds(len, (double)tol, &lo2, &hi2);
  if (lo2_hi2) {
    lo2_hi2[0] = lo2;
    lo2_hi2[1] = hi2;
  }
  ShellHost sh;
  build_shell(lo2, hi2, &sh);
  const int n = (int)sh.off.size();
  for (int i = 0; i < n && i < cap && offs_out; ++i) {
    offs_out[3 * i] = unpack_x(sh.off[i]);
    offs_out[3 * i + 1] = unpack_y(sh.off[i]);
    offs_out[3 * i + 2] = unpack_z(sh.off[i]);
  }
  return n;
}

int ik_row_table(int len, float tol, int32_t* R_out, int32_t* offs_out, int32_t* tabr_out, int cap,
                 int32_t* rowsr_out, int rowsr_cap) {
  if (len < 1 || len > IK_MAX_LEN || !(tol >= 0.0f && tol < 1.0f)) return IK_ERR_ARG;
  int lo2, hi2;
  shell_bounds(len, (double)tol, &lo2, &hi2);
  ShellHost sh;
  build_shell(lo2, hi2, &sh);
  if (R_out) *R_out = sh.R;
  std::vector<int32_t> tabr, rowsr;
  build_row_table(sh, &tabr, &rowsr);
  if (tabr.empty()) return IK_ERR_UNSUPPORTED;
  const int n = (int)sh.dev_off.size();
  for (int i = 0; i < n && i < cap; ++i) {
    if (offs_out) {
      offs_out[3 * i] = unpack_x(sh.dev_off[i]);
      offs_out[3 * i + 1] = unpack_y(sh.dev_off[i]);
      offs_out[3 * i + 2] = unpack_z(sh.dev_off[i]);
    }
    if (tabr_out) tabr_out[i] = tabr[i];
  }
  for (int i = 0; i < (int)rowsr.size() && i < rowsr_cap && rowsr_out; ++i) rowsr_out[i] = rowsr[i];
  return n;
}

int ik_row_mask_table(int len, float tol, int32_t* sc_start_out, int cap_off, int32_t* sctabr_out, int cap_sc) {
  if (len < 1 || len > IK_MAX_LEN || !(tol >= 0.0f && tol < 1.0f)) return IK_ERR_ARG;
  int lo2, hi2;
  shell_bounds(len, (double)tol, &lo2, &hi2);
  ShellHost sh;
  build_shell(lo2, hi2, &sh);
  std::vector<int32_t> sctabr;
  build_row_mask_table(sh, &sctabr);
  if (sctabr.empty()) return IK_ERR_UNSUPPORTED;
  for (int i = 0; i <= (int)sh.dev_off.size() && i < cap_off && sc_start_out; ++i) sc_start_out[i] = sh.sc_start[i];
  for (int i = 0; i < (int)sctabr.size() && i < cap_sc && sctabr_out; ++i) sctabr_out[i] = sctabr[i];
  return (int)sctabr.size();
}

int ik_supercover_offsets(const int32_t d[3], int32_t* vox_out, int cap) {
  if (!d) return IK_ERR_ARG;
  for (int i = 0; i < 3; ++i)
    if (d[i] < -127 || d[i] > 127) return IK_ERR_ARG;
  std::vector<int32_t> sc;
  supercover_traverse(d[0], d[1], d[2], &sc);
  const int n = (int)sc.size();
  for (int i = 0; i < n && i < cap && vox_out; ++i) {
    vox_out[3 * i] = unpack_x(sc[i]);
    vox_out[3 * i + 1] = unpack_y(sc[i]);
    vox_out[3 * i + 2] = unpack_z(sc[i]);
  }
  return n;
}

}  // extern "C"
