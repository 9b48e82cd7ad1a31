// Uneven batches: many independent reach + path problems, each with its own
// grid, obstacles, arm, root, target and waypoint count, solved together.
//
// Problems run through K lanes (a CUDA stream plus device buffers sized for
// the largest problem); lane l takes problems l, l + K, ...  Every problem is
// the same launch sequence as a single reach + path (rasterise, forward sets,
// reach, waypoint survivor sets, smooth chain) with its own dimensions,
// tiling and shell tables; segment tests walk the supercover on the fly, as
// a grid solved once does not repay building edge masks.  Shell tables are
// built once per distinct segment length and shared by every problem.  The
// whole batch is recorded as one CUDA graph (one branch per lane, joined at
// the end) and launched once.  The lane count and the tile depth come from
// the autotuner below unless the caller fixes them.

#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <map>
#include <utility>
#include <vector>

#include "ik_internal.h"

using namespace ikb;

namespace {

struct DevArr {
  void* p = nullptr;
  size_t bytes = 0;
};

// Device tables of one shell for one tiling (tab/sctab depend on it).
struct BatchShell {
  ShellHost host;
  int32_t *off = nullptr, *rows = nullptr, *sc_start = nullptr, *sc = nullptr;
  std::map<std::pair<int, int>, std::pair<int32_t*, int32_t*>> tabs;  // (P, TY) -> (tab, sctab)
};

struct Lane {
  cudaStream_t st = nullptr;
  DevArr occ, F, Fbox, V, Vbox, Vw, Vwbox, g, eps, chain, boxes, pts;
};

struct ProbInfo {
  Dims d;
  TileCfg tc;
  TileCfg tcs[IK_MAX_SEG];  // per segment: tc, or a narrower pitch where tc's halos do not fit
  ArmDev arm;
  int S, W;
  size_t off_reach, off_poses, off_relax;  // into the packed outputs (int32 units)
  size_t off_boxes;                         // into the packed device boxes
  int n_boxes;
};

int cu(cudaError_t e) { return e == cudaSuccess ? IK_OK : (e == cudaErrorMemoryAllocation ? IK_ERR_OOM : IK_ERR_CUDA); }

#define CKB(call)                        \
  do {                                   \
    int _r = cu(call);                   \
    if (_r) return _r;                   \
  } while (0)

int alloc(DevArr& a, size_t bytes, bool zero = false) {
  bytes = std::max<size_t>(bytes, 16);
  if (a.bytes >= bytes) return IK_OK;
  cudaFree(a.p);
  a.p = nullptr;
  a.bytes = 0;
  CKB(cudaMalloc(&a.p, bytes));
  a.bytes = bytes;
  if (zero) CKB(cudaMemset(a.p, 0, bytes));
  return IK_OK;
}

template <typename T>
T* P(DevArr& a) {
  return reinterpret_cast<T*>(a.p);
}

struct Engine {
  std::map<std::pair<int, int>, BatchShell*> shells;
  std::vector<Lane> lanes;
  DevArr boxes_all, out_reach, out_found, out_poses, out_relax, out_status, roots, targets;

  ~Engine() {
    for (auto& kv : shells) {
      BatchShell* s = kv.second;
      cudaFree(s->off);
      cudaFree(s->rows);
      cudaFree(s->sc_start);
      cudaFree(s->sc);
      for (auto& t : s->tabs) {
        cudaFree(t.second.first);
        cudaFree(t.second.second);
      }
      delete s;
    }
    for (Lane& l : lanes) {
      DevArr* a[] = {&l.occ, &l.F, &l.Fbox, &l.V, &l.Vbox, &l.Vw, &l.Vwbox, &l.g, &l.eps, &l.chain, &l.boxes, &l.pts};
      for (DevArr* x : a) cudaFree(x->p);
      if (l.st) cudaStreamDestroy(l.st);
    }
    DevArr* o[] = {&boxes_all, &out_reach, &out_found, &out_poses, &out_relax, &out_status, &roots, &targets};
    for (DevArr* x : o) cudaFree(x->p);
  }

  int shell(int lo2, int hi2, BatchShell** out) {
    auto key = std::make_pair(lo2, hi2);
    auto it = shells.find(key);
    if (it != shells.end()) {
      *out = it->second;
      return IK_OK;
    }
    BatchShell* s = new BatchShell();
    shells[key] = s;
    build_shell(lo2, hi2, &s->host);
    const size_t n = s->host.dev_off.size();
    if (n == 0) return IK_ERR_ARG;
    CKB(cudaMalloc(&s->off, n * 4));
    CKB(cudaMalloc(&s->rows, s->host.rows.size() * 4));
    CKB(cudaMalloc(&s->sc_start, (n + 1) * 4));
    CKB(cudaMalloc(&s->sc, s->host.sc.size() * 4));
    CKB(cudaMemcpy(s->off, s->host.dev_off.data(), n * 4, cudaMemcpyHostToDevice));
    CKB(cudaMemcpy(s->rows, s->host.rows.data(), s->host.rows.size() * 4, cudaMemcpyHostToDevice));
    CKB(cudaMemcpy(s->sc_start, s->host.sc_start.data(), (n + 1) * 4, cudaMemcpyHostToDevice));
    CKB(cudaMemcpy(s->sc, s->host.sc.data(), s->host.sc.size() * 4, cudaMemcpyHostToDevice));
    *out = s;
    return IK_OK;
  }

  // tab / sctab of a shell for a tiling (same encoding as the grid API)
  int tables(BatchShell* s, const TileCfg& tc, int32_t** tab, int32_t** sctab) {
    auto key = std::make_pair(tc.P, tc.TY);
    auto it = s->tabs.find(key);
    if (it == s->tabs.end()) {
      const size_t n = s->host.dev_off.size();
      std::vector<int32_t> t(n), st(s->host.sc.size());
      for (size_t i = 0; i < n; ++i) {
        const int32_t o = s->host.dev_off[i];
        const int delta = unpack_y(o) * tc.P + (unpack_x(o) >> 5);
        t[i] = (int32_t)(((uint32_t)delta << 5) | (uint32_t)(unpack_x(o) & 31));
      }
      const int RY = tc.TY + 2 * s->host.R;
      for (size_t i = 0; i < st.size(); ++i) {
        const int32_t v = s->host.sc[i];
        const int delta = (unpack_z(v) * RY + unpack_y(v)) * tc.P + (unpack_x(v) >> 5);
        st[i] = (int32_t)(((uint32_t)delta << 5) | (uint32_t)(unpack_x(v) & 31));
      }
      int32_t *dt = nullptr, *ds = nullptr;
      CKB(cudaMalloc(&dt, n * 4));
      CKB(cudaMalloc(&ds, std::max<size_t>(st.size(), 1) * 4));
      CKB(cudaMemcpy(dt, t.data(), n * 4, cudaMemcpyHostToDevice));
      CKB(cudaMemcpy(ds, st.data(), st.size() * 4, cudaMemcpyHostToDevice));
      it = s->tabs.emplace(key, std::make_pair(dt, ds)).first;
    }
    *tab = it->second.first;
    *sctab = it->second.second;
    return IK_OK;
  }
};

// One problem's full launch sequence on its lane's stream.
int enqueue_problem(Engine& E, Lane& L, const ProbInfo& pi, int idx, const ik_batch_params& bp) {
  const Dims& d = pi.d;
  const int S = pi.S, W = pi.W;
  const long qs = (long)(S + 1) * d.nw;
  cudaStream_t st = L.st;
  uint32_t* occ = P<uint32_t>(L.occ);
  ArmDev ad = pi.arm;
  for (int k = 0; k < S; ++k) {
    ad.seg[k].occ = occ;
    ad.segf[k] = ad.seg[k];  // whole shells: symmetric
  }
  const int32_t* root = P<int32_t>(E.roots) + 3 * idx;
  const int32_t* target = P<int32_t>(E.targets) + 3 * idx;
  int32_t* reach = P<int32_t>(E.out_reach) + pi.off_reach;
  int32_t* found = P<int32_t>(E.out_found) + idx;
  int32_t* poses = P<int32_t>(E.out_poses) + pi.off_poses;
  int32_t* relax = P<int32_t>(E.out_relax) + pi.off_relax;
  int32_t* status = P<int32_t>(E.out_status) + idx;
  CKB(launch_rasterize(d, P<int32_t>(E.boxes_all) + pi.off_boxes, pi.n_boxes, occ, st));
  // forward sets
  uint32_t* F = P<uint32_t>(L.F);
  int32_t* fb = P<int32_t>(L.Fbox);
  CKB(cudaMemsetAsync(fb, kBoxEmptyByte, (size_t)(S + 1) * 24, st));
  CKB(launch_seed_points(d, root, 1, nullptr, occ, F, d.nw, nullptr, fb, 0, st));
  for (int k = 1; k <= S; ++k)
    CKB(launch_propagate(d, pi.tcs[k - 1], ad.segf[k - 1], F + (k - 1) * d.nw, 0, nullptr, 0, occ, F + k * d.nw,
                         0, 1, fb + 6 * (k - 1), fb + 6 * k, 0, st));
  // reach
  uint32_t* V = P<uint32_t>(L.V);
  int32_t* vb = P<int32_t>(L.Vbox);
  CKB(cudaMemsetAsync(vb, kBoxEmptyByte, (size_t)(S + 1) * 24, st));
  CKB(launch_seed_points(d, target, 1, F + (long)S * d.nw, nullptr, V + (long)S * d.nw, qs, nullptr,
                         vb + 6 * S, 0, st));
  for (int k = S; k >= 1; --k)
    CKB(launch_propagate(d, pi.tcs[k - 1], ad.seg[k - 1], V + (long)k * d.nw, 0, F + (long)(k - 1) * d.nw, 0,
                         occ, V + (long)(k - 1) * d.nw, 0, 1, vb + 6 * k, vb + 6 * (k - 1), 0, st));
  CKB(launch_traceback(d, ad, root, V, qs, 1, reach, found, st));
  // waypoint survivor sets
  uint32_t* Vw = P<uint32_t>(L.Vw);
  int32_t* wb = P<int32_t>(L.Vwbox);
  CKB(cudaMemsetAsync(wb, kBoxEmptyByte, (size_t)W * (S + 1) * 24, st));
  CKB(cudaMemset2DAsync(Vw + (long)S * d.nw, (size_t)qs * 4, 0, (size_t)d.nw * 4, (size_t)W, st));
  CKB(launch_guide_targets(d, ad, occ, F + (long)S * d.nw, reach, found, 1, W, 0, bp.eps2, bp.eps2_max,
                           P<int32_t>(L.g), P<int32_t>(L.eps), Vw, wb, st));
  for (int k = S; k >= 1; --k)
    CKB(launch_propagate(d, pi.tcs[k - 1], ad.seg[k - 1], Vw + (long)k * d.nw, qs, F + (long)(k - 1) * d.nw, 0,
                         occ, Vw + (long)(k - 1) * d.nw, qs, W, wb + 6 * k, wb + 6 * (k - 1),
                         6L * (S + 1), st));
  // smooth chain
  CKB(cudaMemcpyAsync(poses + (long)(W - 1) * 3 * (S + 1), reach, (size_t)12 * (S + 1),
                      cudaMemcpyDeviceToDevice, st));
  ChainArgs a;
  a.P = 1;
  a.W = W;
  a.c = 0;
  a.mode = 0;
  a.delta = bp.delta;
  a.max_relax = bp.max_relax;
  a.found = found;
  a.Vw = Vw;
  a.eps_used = P<int32_t>(L.eps);
  a.poses = poses;
  a.relax = relax;
  a.status = status;
  a.scratch = P<uint32_t>(L.chain);
  a.relaxed_eps_base = bp.eps2;
  CKB(launch_smooth_chain(d, ad, a, st));
  return IK_OK;
}

int check_problem(const ik_problem& p) {
  if (p.nx < 32 || p.nx > 1024 || p.nx % 32 || p.ny < 1 || p.ny > 1024 || p.nz < 1 || p.nz > 1024)
    return IK_ERR_ARG;
  if (p.n_seg < 1 || p.n_seg > IK_MAX_SEG || !p.len || !(p.tol >= 0.f && p.tol < 1.f)) return IK_ERR_ARG;
  for (int k = 0; k < p.n_seg; ++k)
    if (p.len[k] < 1 || p.len[k] > IK_MAX_LEN) return IK_ERR_ARG;
  if (p.n_way < 2 || p.n_way > 4096 || p.n_boxes < 0 || (p.n_boxes > 0 && !p.boxes)) return IK_ERR_ARG;
  for (int i = 0; i < 3; ++i) {
    const int ext = i == 0 ? p.nx : (i == 1 ? p.ny : p.nz);
    if (p.root[i] < 0 || p.root[i] >= ext || p.target[i] < 0 || p.target[i] >= ext) return IK_ERR_ARG;
  }
  return IK_OK;
}

}  // namespace

extern "C" {

int ik_batch_output_sizes(const ik_problem* probs, int n, size_t* reach_ints, size_t* poses_ints,
                          size_t* relax_ints) {
  if (n < 0 || (n > 0 && !probs)) return IK_ERR_ARG;
  size_t r = 0, p = 0, x = 0;
  for (int i = 0; i < n; ++i) {
    r += 3 * (size_t)(probs[i].n_seg + 1);
    p += 3 * (size_t)(probs[i].n_seg + 1) * probs[i].n_way;
    x += 2 * (size_t)probs[i].n_way;
  }
  if (reach_ints) *reach_ints = r;
  if (poses_ints) *poses_ints = p;
  if (relax_ints) *relax_ints = x;
  return IK_OK;
}

int ik_solve_batch(const ik_problem* probs, int n, const ik_batch_params* bp, int32_t* found_out,
                   int32_t* reach_out, int32_t* poses_out, int32_t* relax_out, int32_t* status_out,
                   double* gpu_ms_out) {
  if (n < 0 || (n > 0 && (!probs || !found_out || !reach_out || !poses_out || !relax_out ||
                          !status_out)) || !bp)
    return IK_ERR_ARG;
  if (bp->delta < 0 || bp->delta > 4096 || bp->eps2 < 0 || bp->eps2 > 4096 || bp->eps2_max < 0 ||
      bp->eps2_max > 4096 || bp->max_relax < -1 || bp->lanes < 0 || bp->lanes > 256)
    return IK_ERR_ARG;
  if (n == 0) return IK_OK;
  for (int i = 0; i < n; ++i) {
    int rc = check_problem(probs[i]);
    if (rc) return rc;
  }
  int rc = cu(set_kernel_attributes());
  if (rc) return rc;
  Engine E;
  std::vector<ProbInfo> info(n);
  size_t r_ints = 0, p_ints = 0, x_ints = 0, b_ints = 0;
  size_t max_nw = 0, max_qs = 0, max_vw = 0, max_boxes = 0, max_sp1 = 0, max_w = 0;
  std::vector<int32_t> roots(3 * n), targets(3 * n);
  for (int i = 0; i < n; ++i) {
    const ik_problem& p = probs[i];
    ProbInfo& pi = info[i];
    pi.d.nx = p.nx;
    pi.d.ny = p.ny;
    pi.d.nz = p.nz;
    pi.d.wx = p.nx / 32;
    pi.d.nw = (long)pi.d.wx * p.ny * p.nz;
    pi.tc = make_tile_cfg(pi.d);
    pi.S = p.n_seg;
    pi.W = p.n_way;
    memset(&pi.arm, 0, sizeof(pi.arm));
    pi.arm.S = p.n_seg;
    for (int k = 0; k < p.n_seg; ++k) {
      int lo2, hi2;
      shell_bounds(p.len[k], (double)p.tol, &lo2, &hi2);
      if (hi2 < lo2) return IK_ERR_ARG;
      BatchShell* s = nullptr;
      if ((rc = E.shell(lo2, hi2, &s))) return rc;
      // Without edge masks the tiled kernel stages an occupancy halo beside
      // the source halo; where both do not fit at the grid's pitch, the
      // narrowest pitch (row width + 2 words) is taken for this segment.
      TileCfg tck = pi.tc;
      if (tile_occ_smem_bytes(tck, s->host.R) == 0) {
        TileCfg narrow = pi.tc;
        narrow.P = pi.d.wx + 2;
        if (narrow.P <= 31 && tile_occ_smem_bytes(narrow, s->host.R) > 0) tck = narrow;
      }
      pi.tcs[k] = tck;
      int32_t *tab = nullptr, *sctab = nullptr;
      if ((rc = E.tables(s, tck, &tab, &sctab))) return rc;
      SegDev& sd = pi.arm.seg[k];
      sd.off = s->off;
      sd.rows = s->rows;
      sd.sc_start = s->sc_start;
      sd.sc = s->sc;
      sd.mask = nullptr;
      sd.tab = tab;
      sd.sctab = sctab;
      sd.n = (int)s->host.dev_off.size();
      sd.lo2 = lo2;
      sd.hi2 = hi2;
      sd.R = s->host.R;
      pi.arm.len[k] = p.len[k];
    }
    pi.off_reach = r_ints;
    pi.off_poses = p_ints;
    pi.off_relax = x_ints;
    pi.off_boxes = b_ints;
    pi.n_boxes = p.n_boxes;
    r_ints += 3 * (size_t)(pi.S + 1);
    p_ints += 3 * (size_t)(pi.S + 1) * pi.W;
    x_ints += 2 * (size_t)pi.W;
    b_ints += 6 * (size_t)p.n_boxes;
    const size_t qs = (size_t)(pi.S + 1) * pi.d.nw;
    max_nw = std::max(max_nw, (size_t)pi.d.nw);
    max_qs = std::max(max_qs, qs);
    max_vw = std::max(max_vw, qs * pi.W);
    max_boxes = std::max(max_boxes, (size_t)p.n_boxes);
    max_sp1 = std::max(max_sp1, (size_t)(pi.S + 1));
    max_w = std::max(max_w, (size_t)pi.W);
    memcpy(&roots[3 * i], p.root, 12);
    memcpy(&targets[3 * i], p.target, 12);
  }
  // inputs and outputs for the whole batch
  std::vector<int32_t> boxes(std::max<size_t>(b_ints, 1));
  for (int i = 0; i < n; ++i)
    if (probs[i].n_boxes) memcpy(&boxes[info[i].off_boxes], probs[i].boxes, (size_t)probs[i].n_boxes * 24);
  if ((rc = alloc(E.boxes_all, boxes.size() * 4))) return rc;
  if ((rc = alloc(E.roots, roots.size() * 4))) return rc;
  if ((rc = alloc(E.targets, targets.size() * 4))) return rc;
  if ((rc = alloc(E.out_reach, r_ints * 4))) return rc;
  if ((rc = alloc(E.out_found, (size_t)n * 4))) return rc;
  if ((rc = alloc(E.out_poses, p_ints * 4))) return rc;
  if ((rc = alloc(E.out_relax, x_ints * 4))) return rc;
  if ((rc = alloc(E.out_status, (size_t)n * 4))) return rc;
  CKB(cudaMemcpy(E.boxes_all.p, boxes.data(), boxes.size() * 4, cudaMemcpyHostToDevice));
  CKB(cudaMemcpy(E.roots.p, roots.data(), roots.size() * 4, cudaMemcpyHostToDevice));
  CKB(cudaMemcpy(E.targets.p, targets.data(), targets.size() * 4, cudaMemcpyHostToDevice));
  // lanes: each sized for the largest problem
  int K = bp->lanes > 0 ? bp->lanes : 16;
  K = std::min(K, n);
  E.lanes.resize(K);
  for (Lane& L : E.lanes) {
    CKB(cudaStreamCreateWithFlags(&L.st, cudaStreamNonBlocking));
    if ((rc = alloc(L.occ, max_nw * 4))) return rc;
    if ((rc = alloc(L.F, max_qs * 4))) return rc;
    if ((rc = alloc(L.Fbox, max_sp1 * 24))) return rc;
    if ((rc = alloc(L.V, max_qs * 4))) return rc;
    if ((rc = alloc(L.Vbox, max_sp1 * 24))) return rc;
    if ((rc = alloc(L.Vw, max_vw * 4))) return rc;
    if ((rc = alloc(L.Vwbox, max_w * max_sp1 * 24))) return rc;
    if ((rc = alloc(L.g, max_w * 12))) return rc;
    if ((rc = alloc(L.eps, max_w * 4))) return rc;
    if ((rc = alloc(L.chain, 2 * max_qs * 4, true))) return rc;
  }
  CKB(cudaDeviceSynchronize());
  // record the whole batch as one graph: a root stream forks one branch per
  // lane (problems of a lane run in order), the branches join at the end
  cudaStream_t root_st = nullptr;
  CKB(cudaStreamCreateWithFlags(&root_st, cudaStreamNonBlocking));
  std::vector<cudaEvent_t> ev(K + 1, nullptr);
  for (auto& e : ev) CKB(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  rc = cu(cudaStreamBeginCapture(root_st, cudaStreamCaptureModeThreadLocal));
  if (!rc) {
    rc = cu(cudaEventRecord(ev[K], root_st));
    for (int l = 0; l < K && !rc; ++l) rc = cu(cudaStreamWaitEvent(E.lanes[l].st, ev[K], 0));
    for (int i = 0; i < n && !rc; ++i) rc = enqueue_problem(E, E.lanes[i % K], info[i], i, *bp);
    for (int l = 0; l < K && !rc; ++l) {
      rc = cu(cudaEventRecord(ev[l], E.lanes[l].st));
      if (!rc) rc = cu(cudaStreamWaitEvent(root_st, ev[l], 0));
    }
    cudaError_t e2 = cudaStreamEndCapture(root_st, &graph);
    if (!rc) rc = cu(e2);
  }
  if (!rc) rc = cu(cudaGraphInstantiate(&exec, graph, 0));
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  if (!rc) rc = cu(cudaEventCreate(&t0));
  if (!rc) rc = cu(cudaEventCreate(&t1));
  if (!rc) rc = cu(cudaEventRecord(t0, root_st));
  if (!rc) rc = cu(cudaGraphLaunch(exec, root_st));
  if (!rc) rc = cu(cudaEventRecord(t1, root_st));
  if (!rc) rc = cu(cudaStreamSynchronize(root_st));
  if (!rc && gpu_ms_out) {
    float ms = 0.f;
    rc = cu(cudaEventElapsedTime(&ms, t0, t1));
    *gpu_ms_out = ms;
  }
  if (!rc) rc = cu(cudaMemcpy(found_out, E.out_found.p, (size_t)n * 4, cudaMemcpyDeviceToHost));
  if (!rc) rc = cu(cudaMemcpy(reach_out, E.out_reach.p, r_ints * 4, cudaMemcpyDeviceToHost));
  if (!rc) rc = cu(cudaMemcpy(poses_out, E.out_poses.p, p_ints * 4, cudaMemcpyDeviceToHost));
  if (!rc) rc = cu(cudaMemcpy(relax_out, E.out_relax.p, x_ints * 4, cudaMemcpyDeviceToHost));
  if (!rc) rc = cu(cudaMemcpy(status_out, E.out_status.p, (size_t)n * 4, cudaMemcpyDeviceToHost));
  if (t0) cudaEventDestroy(t0);
  if (t1) cudaEventDestroy(t1);
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  for (auto& e : ev)
    if (e) cudaEventDestroy(e);
  cudaStreamDestroy(root_st);
  return rc;
}

}  // extern "C"
