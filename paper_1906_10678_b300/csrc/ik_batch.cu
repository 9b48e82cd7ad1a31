// Uneven batches: many independent reach + path problems, each with its own
// grid, obstacles, arm, root, target and waypoint count, solved together by
// one persistent launch (k_batch_persistent, see ik_batch_kernel.cuh).
//
// The host builds, per call, one descriptor per problem (dimensions, the
// 16-slice tiling of each segment, pointers into one device pool, where every
// problem owns 128-byte-aligned regions for its occupancy, forward, reach and
// waypoint survivor sets, chain scratch, boxes and small records) and the
// first items (the rasterise slabs of every problem).  The pool is cleared,
// the kernel runs, and its last item per problem copies the results into the
// caller's packed outputs.  Shell tables (per segment length) and their
// shared-memory deltas (per tiling) are built once and kept by the engine, as
// are the pool, the queue and the pinned staging: an engine allocates on the
// first call that needs more memory and reuses it afterwards.  When a batch
// needs more pool than the engine's budget it runs as several launches
// (waves) in problem order.

#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <utility>
#include <vector>

#include "ik_internal.h"

using namespace ikb;

namespace {

int cu(cudaError_t e) {
  if (e == cudaSuccess) return IK_OK;
  note_cuda_error(e);
  cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? IK_ERR_OOM : IK_ERR_CUDA;
}

#define CKB(call)      \
  do {                 \
    int _r = cu(call); \
    if (_r) return _r; \
  } while (0)

struct DevArr {
  void* p = nullptr;
  size_t bytes = 0;
};

// Grow-only device buffer (contents not kept).
int grow(DevArr& a, size_t bytes) {
  bytes = std::max<size_t>(bytes, 256);
  if (a.bytes >= bytes) return IK_OK;
  if (a.p) CKB(cudaFree(a.p));
  a.p = nullptr;
  a.bytes = 0;
  CKB(cudaMalloc(&a.p, bytes));
  a.bytes = bytes;
  return IK_OK;
}

// Device tables of one shell, and its shared-memory deltas per tiling.
struct BatchShell {
  ShellHost host;
  int32_t *off = nullptr, *rows = nullptr, *sc_start = nullptr, *sc = nullptr;
  std::map<std::pair<int, int>, std::pair<int32_t*, int32_t*>> tabs;  // (P, TY) -> (tab, sctab)
};

constexpr size_t kAlignWords = 32;  // 128 bytes
size_t align_words(size_t w) { return (w + kAlignWords - 1) / kAlignWords * kAlignWords; }

// Pool words of one problem (every region rounded to 128 bytes).
struct Layout {
  size_t occ, F, V, Vw, chain, Fbox, Vbox, Vwbox, reach, found, g, eps, poses, relax, status, total;
};

Layout layout_of(const Dims& d, int S, int W) {
  Layout L;
  size_t at = 0;
  auto take = [&](size_t words) {
    const size_t a = at;
    at += align_words(words);
    return a;
  };
  const size_t nw = (size_t)d.nw;
  L.occ = take(nw);
  L.F = take((S + 1) * nw);
  L.V = take((S + 1) * nw);
  L.Vw = take((size_t)W * (S + 1) * nw);
  L.chain = take(2 * (S + 1) * nw);
  L.Fbox = take(6 * (S + 1));
  L.Vbox = take(6 * (S + 1));
  L.Vwbox = take(6 * (S + 1) * (size_t)W);
  L.reach = take(3 * (S + 1));
  L.found = take(1);
  L.g = take(3 * (size_t)W);
  L.eps = take((size_t)W);
  L.poses = take(3 * (S + 1) * (size_t)W);
  L.relax = take(2 * (size_t)W);
  L.status = take(1);
  L.total = at;
  return L;
}

int check_problem(const ik_problem& p) {
  if (p.nx < 32 || p.nx > 1024 || p.nx % 32 || p.ny < 1 || p.ny > 1024 || p.nz < 1 || p.nz > 1024)
    return IK_ERR_ARG;
  if (p.n_seg < 1 || p.n_seg > IK_MAX_SEG || !p.len || !(p.tol >= 0.f && p.tol < 1.f)) return IK_ERR_ARG;
  for (int k = 0; k < p.n_seg; ++k)
    if (p.len[k] < 1 || p.len[k] > IK_MAX_LEN) return IK_ERR_ARG;
  if (p.n_way < 2 || p.n_way > 4096 || p.n_boxes < 0 || p.n_boxes > 8192 || (p.n_boxes > 0 && !p.boxes))
    return IK_ERR_ARG;
  for (int i = 0; i < 3; ++i) {
    const int ext = i == 0 ? p.nx : (i == 1 ? p.ny : p.nz);
    if (p.root[i] < 0 || p.root[i] >= ext || p.target[i] < 0 || p.target[i] >= ext) return IK_ERR_ARG;
  }
  return IK_OK;
}

}  // namespace

struct ik_batch_engine_s {
  int device = 0;
  int num_sms = 148;
  size_t budget = 0;  // pool bytes per launch (0: from the free memory at the first call)
  std::mutex mu;
  std::map<std::pair<int, int>, BatchShell*> shells;
  DevArr pool, descs, items, ctl, state, boxes;
  // host-output form (ik_solve_batch): device outputs kept between calls
  DevArr out_found, out_reach, out_poses, out_relax, out_status, out_rc;
  char* pinned = nullptr;
  size_t pinned_bytes = 0;
  cudaEvent_t staged = nullptr;  // the last upload out of `pinned` is done
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  long long timeout_ns = 20LL * 1000 * 1000 * 1000;
  int pairs = 1;          // ik_batch_engine_set_pairs
  size_t smem_limit = 0;  // batch_smem_limit() of the device, at the first plan

  ~ik_batch_engine_s() {
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(device);
    cudaDeviceSynchronize();
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
    DevArr* all[] = {&pool, &descs, &items, &ctl, &state, &boxes, &out_found, &out_reach, &out_poses,
                     &out_relax, &out_status, &out_rc};
    for (DevArr* a : all) cudaFree(a->p);
    if (pinned) cudaFreeHost(pinned);
    if (staged) cudaEventDestroy(staged);
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    cudaSetDevice(prev);
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

  // tab / sctab of a shell for a tiling (the encoding of the grid API)
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

  int pinned_grow(size_t bytes) {
    if (pinned_bytes >= bytes) return IK_OK;
    if (staged) CKB(cudaEventSynchronize(staged));
    if (pinned) CKB(cudaFreeHost(pinned));
    pinned = nullptr;
    pinned_bytes = 0;
    CKB(cudaMallocHost((void**)&pinned, bytes));
    pinned_bytes = bytes;
    return IK_OK;
  }
};

namespace {

struct ProbPlan {
  Dims d;
  TileCfg tcs[IK_MAX_SEG];
  ArmDev arm;
  Layout lay;
  size_t smem;  // dynamic shared memory its items need
  int n_slabs;
  size_t off_reach, off_poses, off_relax, off_boxes;
};

// Tiling of the persistent kernel for one segment: 16 z slices per tile,
// the grid's row tiling and pitch; where the two halos do not fit, the
// narrowest pitch, then 8 slices.  Returns false when no form fits.
bool batch_tiling(const Dims& d, int R, TileCfg* out) {
  TileCfg tc = make_tile_cfg(d);
  tc.TZ = kBatchTZ;
  tc.tiles_z = (d.nz + tc.TZ - 1) / tc.TZ;
  if (tile_occ_smem_bytes(tc, R) == 0) {
    TileCfg narrow = tc;
    narrow.P = d.wx + 2;
    if (narrow.P <= 31 && tile_occ_smem_bytes(narrow, R) > 0) {
      tc = narrow;
    } else {
      narrow.TZ = 8;
      narrow.tiles_z = (d.nz + 7) / 8;
      if (narrow.P > 31 || tile_occ_smem_bytes(narrow, R) == 0) return false;
      tc = narrow;
    }
  }
  *out = tc;
  return true;
}

int plan_problems(ik_batch_engine_s* E, const ik_problem* probs, int n, std::vector<ProbPlan>* plans) {
  plans->resize(n);
  if (!E->smem_limit) E->smem_limit = batch_smem_limit();
  size_t r = 0, p = 0, x = 0, b = 0;
  for (int i = 0; i < n; ++i) {
    const ik_problem& pr = probs[i];
    ProbPlan& pl = (*plans)[i];
    pl.d.nx = pr.nx;
    pl.d.ny = pr.ny;
    pl.d.nz = pr.nz;
    pl.d.wx = pr.nx / 32;
    pl.d.nw = (long)pl.d.wx * pr.ny * pr.nz;
    memset(&pl.arm, 0, sizeof(pl.arm));
    pl.arm.S = pr.n_seg;
    pl.smem = std::max(batch_chain_smem_bytes(), (size_t)pr.n_boxes * 24);
    for (int k = 0; k < pr.n_seg; ++k) {
      int lo2, hi2;
      shell_bounds(pr.len[k], (double)pr.tol, &lo2, &hi2);
      if (hi2 < lo2) return IK_ERR_ARG;
      BatchShell* s = nullptr;
      int rc = E->shell(lo2, hi2, &s);
      if (rc) return rc;
      if (s->host.R > 31) return IK_ERR_UNSUPPORTED;  // the tiled bodies' x halo is one word
      TileCfg tc;
      if (!batch_tiling(pl.d, s->host.R, &tc)) return IK_ERR_UNSUPPORTED;
      // the level's waypoint queries in pairs (one more halo) where it fits
      const size_t occ_bytes = tile_occ_smem_bytes(tc, s->host.R), pair_bytes = 3 * (occ_bytes / 2);
      tc.pair = E->pairs && pr.n_way >= 2 && pair_bytes <= E->smem_limit ? 1 : 0;
      pl.tcs[k] = tc;
      pl.smem = std::max(pl.smem, tc.pair ? pair_bytes : occ_bytes);
      int32_t *tab = nullptr, *sctab = nullptr;
      if ((rc = E->tables(s, tc, &tab, &sctab))) return rc;
      SegDev& sd = pl.arm.seg[k];
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
      pl.arm.len[k] = pr.len[k];
    }
    pl.lay = layout_of(pl.d, pr.n_seg, pr.n_way);
    pl.n_slabs = (pr.nz + kBatchSlab - 1) / kBatchSlab;
    pl.off_reach = r;
    pl.off_poses = p;
    pl.off_relax = x;
    pl.off_boxes = b;
    r += 3 * (size_t)(pr.n_seg + 1);
    p += 3 * (size_t)(pr.n_seg + 1) * pr.n_way;
    x += 2 * (size_t)pr.n_way;
    b += align_words(6 * (size_t)pr.n_boxes);
  }
  return IK_OK;
}

// Upper bound of the items a problem can push (every tile at every level).
long long item_bound(const ik_problem& p, const ProbPlan& pl) {
  long long c = pl.n_slabs + 4 + p.n_way;
  for (int k = 0; k < p.n_seg; ++k) {
    const long long tiles = (long long)pl.tcs[k].tiles_y * pl.tcs[k].tiles_z;
    c += tiles * (2 + p.n_way);
  }
  return c;
}

// Enqueues problems [lo, hi) as one persistent launch.
// The device descriptor of problem i (index in the caller's arrays) whose
// pool region starts at base and whose boxes go to dboxes (device) through
// hboxes (host staging).
void fill_desc(const ik_problem& p, const ProbPlan& pl, int i, uint32_t* base, int32_t* dboxes, int32_t* hboxes,
               int32_t* found, int32_t* reach, int32_t* poses, int32_t* relax, int32_t* status, int32_t* rc_out,
               BatchProb* out) {
  BatchProb& B = *out;
  memset(&B, 0, sizeof(B));
  B.d = pl.d;
  for (int k = 0; k < IK_MAX_SEG; ++k) B.tcs[k] = pl.tcs[k];
  B.arm = pl.arm;
  B.S = p.n_seg;
  B.W = p.n_way;
  B.n_boxes = p.n_boxes;
  B.n_slabs = pl.n_slabs;
  for (int c = 0; c < 3; ++c) {
    B.root[c] = p.root[c];
    B.target[c] = p.target[c];
  }
  if (p.n_boxes) memcpy(hboxes, p.boxes, (size_t)p.n_boxes * 24);
  B.boxes = dboxes;
  const Layout& L = pl.lay;
  B.occ = base + L.occ;
  B.F = base + L.F;
  B.V = base + L.V;
  B.Vw = base + L.Vw;
  B.chain = base + L.chain;
  B.Fbox = (int32_t*)(base + L.Fbox);
  B.Vbox = (int32_t*)(base + L.Vbox);
  B.Vwbox = (int32_t*)(base + L.Vwbox);
  B.reach = (int32_t*)(base + L.reach);
  B.found = (int32_t*)(base + L.found);
  B.g = (int32_t*)(base + L.g);
  B.eps = (int32_t*)(base + L.eps);
  B.poses = (int32_t*)(base + L.poses);
  B.relax = (int32_t*)(base + L.relax);
  B.status = (int32_t*)(base + L.status);
  for (int k = 0; k < p.n_seg; ++k) {
    B.arm.seg[k].occ = B.occ;
    B.arm.segf[k] = B.arm.seg[k];  // whole shells: symmetric
  }
  B.o_found = found + i;
  B.o_reach = reach + pl.off_reach;
  B.o_poses = poses + pl.off_poses;
  B.o_relax = relax + pl.off_relax;
  B.o_status = status + i;
  B.o_rc = rc_out + i;
}

int run_wave(ik_batch_engine_s* E, const ik_problem* probs, const std::vector<ProbPlan>& plans, int lo, int hi,
             const ik_batch_params* bp, int32_t* found, int32_t* reach, int32_t* poses, int32_t* relax,
             int32_t* status, int32_t* rc_out, cudaStream_t st) {
  const int n = hi - lo;
  size_t pool_words = 0, box_words = 0, smem = 0;
  long long n_items = 0, n_first = 0;
  for (int i = lo; i < hi; ++i) {
    pool_words += plans[i].lay.total;
    box_words += align_words(6 * (size_t)probs[i].n_boxes);
    smem = std::max(smem, plans[i].smem);
    n_items += item_bound(probs[i], plans[i]);
    n_first += plans[i].n_slabs;
  }
  int rc;
  if ((rc = grow(E->pool, pool_words * 4))) return rc;
  if ((rc = grow(E->descs, (size_t)n * sizeof(BatchProb)))) return rc;
  if ((rc = grow(E->items, (size_t)n_items * sizeof(int4)))) return rc;
  if ((rc = grow(E->ctl, 8 * sizeof(unsigned long long)))) return rc;
  if ((rc = grow(E->state, (size_t)n * sizeof(int2)))) return rc;
  if ((rc = grow(E->boxes, std::max<size_t>(box_words, 1) * 4))) return rc;
  if (smem > batch_smem_limit()) return IK_ERR_UNSUPPORTED;
  CKB(batch_set_smem(smem));
  // host staging: descriptors, per-problem state, first items, boxes
  const size_t desc_b = (size_t)n * sizeof(BatchProb), state_b = (size_t)n * sizeof(int2);
  const size_t items_b = (size_t)n_first * sizeof(int4), boxes_b = box_words * 4;
  const size_t o_state = desc_b, o_items = o_state + state_b, o_boxes = o_items + items_b;
  if ((rc = E->pinned_grow(o_boxes + boxes_b + 64))) return rc;
  if (E->staged) CKB(cudaEventSynchronize(E->staged));  // the previous upload has left the staging
  BatchProb* hd = (BatchProb*)E->pinned;
  int2* hs = (int2*)(E->pinned + o_state);
  int4* hi4 = (int4*)(E->pinned + o_items);
  int32_t* hb = (int32_t*)(E->pinned + o_boxes);
  uint32_t* pool = (uint32_t*)E->pool.p;
  int32_t* dboxes = (int32_t*)E->boxes.p;
  size_t pw = 0, bw = 0;
  long long it = 0;
  for (int i = lo; i < hi; ++i) {
    fill_desc(probs[i], plans[i], i, pool + pw, dboxes + bw, hb + bw, found, reach, poses, relax, status, rc_out,
              &hd[i - lo]);
    pw += plans[i].lay.total;
    bw += align_words(6 * (size_t)probs[i].n_boxes);
    hs[i - lo] = make_int2(0, plans[i].n_slabs);
    for (int s = 0; s < plans[i].n_slabs; ++s) hi4[it++] = make_int4(i - lo + 1, 0, s, 0);
  }
  // uploads, cleared pool and queue, then the launch
  CKB(cudaMemcpyAsync(E->descs.p, hd, desc_b, cudaMemcpyHostToDevice, st));
  CKB(cudaMemcpyAsync(E->state.p, hs, state_b, cudaMemcpyHostToDevice, st));
  CKB(cudaMemsetAsync(E->items.p, 0, (size_t)n_items * sizeof(int4), st));
  CKB(cudaMemcpyAsync(E->items.p, hi4, items_b, cudaMemcpyHostToDevice, st));
  if (boxes_b) CKB(cudaMemcpyAsync(E->boxes.p, hb, boxes_b, cudaMemcpyHostToDevice, st));
  if (!E->staged) CKB(cudaEventCreateWithFlags(&E->staged, cudaEventDisableTiming));
  CKB(cudaEventRecord(E->staged, st));
  CKB(cudaMemsetAsync(E->pool.p, 0, pool_words * 4, st));
  unsigned long long ctl0[8] = {0, (unsigned long long)n_first, 0, 0, 0, 0, 0, 0};
  CKB(cudaMemcpyAsync(E->ctl.p, ctl0, sizeof(ctl0), cudaMemcpyHostToDevice, st));  // pageable: copied now
  CKB(launch_fill_i32(rc_out + lo, n, IK_ERR_TIMEOUT, st));
  BatchQueue q;
  q.items = (int4*)E->items.p;
  q.cap = n_items;
  q.ctl = (unsigned long long*)E->ctl.p;
  q.state = (int2*)E->state.p;
  BatchRules r{bp->delta, bp->eps2, bp->eps2_max, bp->max_relax};
  const int per_sm = bp->blocks_per_sm > 0 ? bp->blocks_per_sm : 1;
  CKB(launch_batch_persistent((const BatchProb*)E->descs.p, n, q, r, E->num_sms * per_sm, smem,
                              E->timeout_ns, st));
  return IK_OK;
}

int solve_async(ik_batch_engine_s* E, const ik_problem* probs, int n, const ik_batch_params* bp,
                int32_t* found, int32_t* reach, int32_t* poses, int32_t* relax, int32_t* status, int32_t* rc_out,
                cudaStream_t st) {
  std::vector<ProbPlan> plans;
  int rc = plan_problems(E, probs, n, &plans);
  if (rc) return rc;
  if (E->budget == 0) {
    size_t fr = 0, tot = 0;
    CKB(cudaMemGetInfo(&fr, &tot));
    E->budget = (size_t)(0.7 * (double)fr);
  }
  // waves: problems in order, each wave's pool within the budget
  int lo = 0;
  while (lo < n) {
    size_t words = plans[lo].lay.total;
    int hi = lo + 1;
    while (hi < n && (words + plans[hi].lay.total) * 4 <= E->budget) words += plans[hi++].lay.total;
    if ((rc = run_wave(E, probs, plans, lo, hi, bp, found, reach, poses, relax, status, rc_out, st)))
      return rc;
    lo = hi;
  }
  return IK_OK;
}

int check_params(const ik_batch_params* bp) {
  if (!bp) return IK_ERR_ARG;
  if (bp->delta < 0 || bp->delta > 4096 || bp->eps2 < 0 || bp->eps2 > 4096 || bp->eps2_max < 0 ||
      bp->eps2_max > 4096 || bp->max_relax < -1 || bp->blocks_per_sm < 0 || bp->blocks_per_sm > 1)
    return IK_ERR_ARG;
  return IK_OK;
}

// The engine behind ik_solve_batch, one per device, kept for the process.
std::mutex g_default_mu;
ik_batch_engine_s* g_default[64] = {nullptr};

}  // namespace

extern "C" {

// A captured uneven batch: its own pool, queue and descriptors, the initial
// queue state kept on the device, and the graph that resets the queue,
// clears the pool and runs the persistent kernel.
struct ik_batch_graph_s {
  int device = 0;
  DevArr pool, descs, items, ctl, state, boxes, items0, state0, ctl0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;

  ~ik_batch_graph_s() {
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(device);
    cudaDeviceSynchronize();
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    DevArr* all[] = {&pool, &descs, &items, &ctl, &state, &boxes, &items0, &state0, &ctl0};
    for (DevArr* a : all) cudaFree(a->p);
    cudaSetDevice(prev);
  }
};

namespace {

// Plans the batch, uploads its descriptors, boxes and initial queue into
// the graph's buffers (synchronously, outside any capture) and captures the
// launch sequence on a private stream.
int capture_uneven(ik_batch_engine_s* E, const ik_problem* probs, int n, const ik_batch_params* bp,
                   int32_t* found, int32_t* reach, int32_t* poses, int32_t* relax, int32_t* status,
                   int32_t* rc_out, ik_batch_graph_s* G) {
  std::vector<ProbPlan> plans;
  int rc = plan_problems(E, probs, n, &plans);
  if (rc) return rc;
  if (E->budget == 0) {
    size_t fr = 0, tot = 0;
    CKB(cudaMemGetInfo(&fr, &tot));
    E->budget = (size_t)(0.7 * (double)fr);
  }
  size_t pool_words = 0, box_words = 0, smem = 0;
  long long n_items = 0, n_first = 0;
  for (int i = 0; i < n; ++i) {
    pool_words += plans[i].lay.total;
    box_words += align_words(6 * (size_t)probs[i].n_boxes);
    smem = std::max(smem, plans[i].smem);
    n_items += item_bound(probs[i], plans[i]);
    n_first += plans[i].n_slabs;
  }
  if (smem > batch_smem_limit() || pool_words * 4 > E->budget) return IK_ERR_UNSUPPORTED;
  if ((rc = grow(G->pool, pool_words * 4))) return rc;
  if ((rc = grow(G->descs, (size_t)n * sizeof(BatchProb)))) return rc;
  if ((rc = grow(G->items, (size_t)n_items * sizeof(int4)))) return rc;
  if ((rc = grow(G->items0, (size_t)n_first * sizeof(int4)))) return rc;
  if ((rc = grow(G->ctl, 8 * sizeof(unsigned long long)))) return rc;
  if ((rc = grow(G->ctl0, 8 * sizeof(unsigned long long)))) return rc;
  if ((rc = grow(G->state, (size_t)n * sizeof(int2)))) return rc;
  if ((rc = grow(G->state0, (size_t)n * sizeof(int2)))) return rc;
  if ((rc = grow(G->boxes, std::max<size_t>(box_words, 1) * 4))) return rc;
  CKB(batch_set_smem(smem));
  std::vector<BatchProb> hd(n);
  std::vector<int2> hs(n);
  std::vector<int4> hi4((size_t)n_first);
  std::vector<int32_t> hb(std::max<size_t>(box_words, 1));
  uint32_t* pool = (uint32_t*)G->pool.p;
  int32_t* dboxes = (int32_t*)G->boxes.p;
  size_t pw = 0, bw = 0;
  long long it = 0;
  for (int i = 0; i < n; ++i) {
    fill_desc(probs[i], plans[i], i, pool + pw, dboxes + bw, hb.data() + bw, found, reach, poses, relax, status,
              rc_out, &hd[i]);
    pw += plans[i].lay.total;
    bw += align_words(6 * (size_t)probs[i].n_boxes);
    hs[i] = make_int2(0, plans[i].n_slabs);
    for (int s = 0; s < plans[i].n_slabs; ++s) hi4[it++] = make_int4(i + 1, 0, s, 0);
  }
  const unsigned long long ctl0[8] = {0, (unsigned long long)n_first, 0, 0, 0, 0, 0, 0};
  CKB(cudaMemcpy(G->descs.p, hd.data(), (size_t)n * sizeof(BatchProb), cudaMemcpyHostToDevice));
  CKB(cudaMemcpy(G->boxes.p, hb.data(), hb.size() * 4, cudaMemcpyHostToDevice));
  CKB(cudaMemcpy(G->state0.p, hs.data(), (size_t)n * sizeof(int2), cudaMemcpyHostToDevice));
  CKB(cudaMemcpy(G->items0.p, hi4.data(), hi4.size() * sizeof(int4), cudaMemcpyHostToDevice));
  CKB(cudaMemcpy(G->ctl0.p, ctl0, sizeof(ctl0), cudaMemcpyHostToDevice));
  BatchQueue q;
  q.items = (int4*)G->items.p;
  q.cap = n_items;
  q.ctl = (unsigned long long*)G->ctl.p;
  q.state = (int2*)G->state.p;
  BatchRules r{bp->delta, bp->eps2, bp->eps2_max, bp->max_relax};
  const int per_sm = bp->blocks_per_sm > 0 ? bp->blocks_per_sm : 1;
  cudaStream_t cs = nullptr;
  CKB(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaMemcpyAsync(G->state.p, G->state0.p, (size_t)n * sizeof(int2), cudaMemcpyDeviceToDevice, cs);
    cudaMemsetAsync(G->items.p, 0, (size_t)n_items * sizeof(int4), cs);
    cudaMemcpyAsync(G->items.p, G->items0.p, hi4.size() * sizeof(int4), cudaMemcpyDeviceToDevice, cs);
    cudaMemcpyAsync(G->ctl.p, G->ctl0.p, sizeof(ctl0), cudaMemcpyDeviceToDevice, cs);
    cudaMemsetAsync(G->pool.p, 0, pool_words * 4, cs);
    launch_fill_i32(rc_out, n, IK_ERR_TIMEOUT, cs);
    launch_batch_persistent((const BatchProb*)G->descs.p, n, q, r, E->num_sms * per_sm, smem, E->timeout_ns, cs);
    const cudaError_t e2 = cudaStreamEndCapture(cs, &G->graph);
    e = e2 != cudaSuccess ? e2 : cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&G->exec, G->graph, 0);
  cudaStreamDestroy(cs);
  return cu(e);
}

}  // namespace

int ik_batch_engine_create(ik_batch_engine* out) {
  if (!out) return IK_ERR_ARG;
  *out = nullptr;
  ik_batch_engine_s* E = new ik_batch_engine_s();
  if (cudaGetDevice(&E->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&E->num_sms, cudaDevAttrMultiProcessorCount, E->device) != cudaSuccess) {
    cudaGetLastError();
    delete E;
    return IK_ERR_CUDA;
  }
  *out = E;
  return IK_OK;
}

int ik_batch_engine_destroy(ik_batch_engine e) {
  delete e;
  return IK_OK;
}

int ik_batch_engine_set_budget(ik_batch_engine e, size_t pool_bytes) {
  if (!e) return IK_ERR_ARG;
  std::lock_guard<std::mutex> lock(e->mu);
  e->budget = pool_bytes;
  return IK_OK;
}

int ik_batch_engine_set_timeout(ik_batch_engine e, int64_t ns) {
  if (!e || ns < 1000) return IK_ERR_ARG;
  std::lock_guard<std::mutex> lock(e->mu);
  e->timeout_ns = ns;
  return IK_OK;
}

int ik_batch_engine_set_pairs(ik_batch_engine e, int on) {
  if (!e || (on != 0 && on != 1)) return IK_ERR_ARG;
  std::lock_guard<std::mutex> lock(e->mu);
  e->pairs = on;
  return IK_OK;
}

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

int ik_solve_batch_async(ik_batch_engine e, const ik_problem* probs, int n, const ik_batch_params* bp,
                         int32_t* found_dev, int32_t* reach_dev, int32_t* poses_dev, int32_t* relax_dev,
                         int32_t* status_dev, int32_t* job_rc_dev, void* cuda_stream) {
  if (!e || n < 0 || (n > 0 && (!probs || !found_dev || !reach_dev || !poses_dev || !relax_dev ||
                                !status_dev || !job_rc_dev)))
    return IK_ERR_ARG;
  int rc = check_params(bp);
  if (rc) return rc;
  for (int i = 0; i < n; ++i)
    if ((rc = check_problem(probs[i]))) return rc;
  if (n == 0) return IK_OK;
  std::lock_guard<std::mutex> lock(e->mu);
  int prev = 0;
  if (cudaGetDevice(&prev) != cudaSuccess) return cu(cudaGetLastError());
  if (prev != e->device) CKB(cudaSetDevice(e->device));
  rc = solve_async(e, probs, n, bp, found_dev, reach_dev, poses_dev, relax_dev, status_dev, job_rc_dev,
                   (cudaStream_t)cuda_stream);
  if (prev != e->device) cudaSetDevice(prev);
  return rc;
}

int ik_solve_batch(const ik_problem* probs, int n, const ik_batch_params* bp, int32_t* found_out,
                   int32_t* reach_out, int32_t* poses_out, int32_t* relax_out, int32_t* status_out,
                   double* gpu_ms_out) {
  if (n < 0 || (n > 0 && (!probs || !found_out || !reach_out || !poses_out || !relax_out || !status_out)))
    return IK_ERR_ARG;
  int rc = check_params(bp);
  if (rc) return rc;
  for (int i = 0; i < n; ++i)
    if ((rc = check_problem(probs[i]))) return rc;
  if (n == 0) return IK_OK;
  int dev = 0;
  CKB(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return IK_ERR_UNSUPPORTED;
  ik_batch_engine_s* E = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_default_mu);
    if (!g_default[dev]) {
      ik_batch_engine eng = nullptr;
      if ((rc = ik_batch_engine_create(&eng))) return rc;
      g_default[dev] = eng;
    }
    E = g_default[dev];
  }
  std::lock_guard<std::mutex> lock(E->mu);
  size_t r_ints = 0, p_ints = 0, x_ints = 0;
  ik_batch_output_sizes(probs, n, &r_ints, &p_ints, &x_ints);
  if ((rc = grow(E->out_found, (size_t)n * 4)) || (rc = grow(E->out_status, (size_t)n * 4)) ||
      (rc = grow(E->out_rc, (size_t)n * 4)) || (rc = grow(E->out_reach, r_ints * 4)) ||
      (rc = grow(E->out_poses, p_ints * 4)) || (rc = grow(E->out_relax, x_ints * 4)))
    return rc;
  if (!E->t0) CKB(cudaEventCreate(&E->t0));
  if (!E->t1) CKB(cudaEventCreate(&E->t1));
  cudaStream_t st = nullptr;
  CKB(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  int32_t* d_rc = (int32_t*)E->out_rc.p;
  rc = cu(cudaEventRecord(E->t0, st));
  if (!rc)
    rc = solve_async(E, probs, n, bp, (int32_t*)E->out_found.p, (int32_t*)E->out_reach.p,
                     (int32_t*)E->out_poses.p, (int32_t*)E->out_relax.p, (int32_t*)E->out_status.p, d_rc, st);
  if (!rc) rc = cu(cudaEventRecord(E->t1, st));
  if (!rc) rc = cu(cudaStreamSynchronize(st));
  if (!rc && gpu_ms_out) {
    float ms = 0.f;
    rc = cu(cudaEventElapsedTime(&ms, E->t0, E->t1));
    *gpu_ms_out = ms;
  }
  std::vector<int32_t> jrc(n, IK_OK);
  if (!rc) rc = cu(cudaMemcpy(jrc.data(), d_rc, (size_t)n * 4, cudaMemcpyDeviceToHost));
  if (!rc) rc = cu(cudaMemcpy(found_out, E->out_found.p, (size_t)n * 4, cudaMemcpyDeviceToHost));
  if (!rc) rc = cu(cudaMemcpy(reach_out, E->out_reach.p, r_ints * 4, cudaMemcpyDeviceToHost));
  if (!rc) rc = cu(cudaMemcpy(poses_out, E->out_poses.p, p_ints * 4, cudaMemcpyDeviceToHost));
  if (!rc) rc = cu(cudaMemcpy(relax_out, E->out_relax.p, x_ints * 4, cudaMemcpyDeviceToHost));
  if (!rc) rc = cu(cudaMemcpy(status_out, E->out_status.p, (size_t)n * 4, cudaMemcpyDeviceToHost));
  cudaStreamDestroy(st);
  if (!rc)
    for (int i = 0; i < n; ++i)
      if (jrc[i] != IK_OK) return jrc[i];
  return rc;
}

}  // extern "C"

int ik_batch_capture_uneven(ik_batch_engine e, const ik_problem* probs, int n, const ik_batch_params* bp,
                            int32_t* found_dev, int32_t* reach_dev, int32_t* poses_dev, int32_t* relax_dev,
                            int32_t* status_dev, int32_t* job_rc_dev, ik_batch_graph* out) {
  if (!e || !out || n <= 0 || !probs || !found_dev || !reach_dev || !poses_dev || !relax_dev || !status_dev ||
      !job_rc_dev)
    return IK_ERR_ARG;
  *out = nullptr;
  int rc = check_params(bp);
  if (rc) return rc;
  for (int i = 0; i < n; ++i)
    if ((rc = check_problem(probs[i]))) return rc;
  std::lock_guard<std::mutex> lock(e->mu);
  int prev = 0;
  if (cudaGetDevice(&prev) != cudaSuccess) return cu(cudaGetLastError());
  if (prev != e->device) CKB(cudaSetDevice(e->device));
  ik_batch_graph_s* G = new ik_batch_graph_s;
  G->device = e->device;
  rc = capture_uneven(e, probs, n, bp, found_dev, reach_dev, poses_dev, relax_dev, status_dev, job_rc_dev, G);
  if (rc) delete G;
  else *out = G;
  if (prev != e->device) cudaSetDevice(prev);
  return rc;
}

int ik_batch_graph_launch(ik_batch_graph g, void* cuda_stream) {
  if (!g || !g->exec) return IK_ERR_ARG;
  int prev = 0;
  if (cudaGetDevice(&prev) != cudaSuccess) return cu(cudaGetLastError());
  if (prev != g->device) CKB(cudaSetDevice(g->device));
  const int rc = cu(cudaGraphLaunch(g->exec, (cudaStream_t)cuda_stream));
  if (prev != g->device) cudaSetDevice(prev);
  return rc;
}

int ik_batch_graph_destroy(ik_batch_graph g) {
  delete g;
  return IK_OK;
}
