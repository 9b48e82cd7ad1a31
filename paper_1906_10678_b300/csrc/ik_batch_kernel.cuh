// The persistent uneven-batch kernel (declared in ik_internal.h; included by
// ik_kernels.cu so that it can call the block-level bodies defined there).
//
// Stages of problem i with S segments and W waypoints, in order:
//   0               rasterise its boxes, one item per slab of 16 z slices
//   1               forward seed F_0 = {root} (and every box of the problem set empty)
//   2 .. S+1        forward level k = t - 1: F_k = D_k(F_{k-1}), items per tile
//   S+2             reach seed V_S = {target} & F_S
//   S+3 .. 2S+2     reach level k = 2S+3 - t: V_{k-1} = F_{k-1} & D_k(V_k), items per tile
//   2S+3            traceback of the reach pose (the minimum-index rule)
//   2S+4            guide point and target set of every waypoint, one item per waypoint
//   2S+5 .. 3S+4    waypoint level k = 3S+5 - t, items per (tile, waypoint)
//   3S+5            the smooth chain of the path, then the outputs are copied out
//   3S+6            done
// Every rule is the grid API's: the same block bodies run here.

enum BatchKind { BK_RASTER, BK_FSEED, BK_FPROP, BK_VSEED, BK_VPROP, BK_TRACE, BK_GUIDE, BK_WPROP, BK_CHAIN,
                 BK_DONE };

__device__ __forceinline__ BatchKind batch_kind(int S, int t, int* k) {
  *k = 0;
  if (t == 0) return BK_RASTER;
  if (t == 1) return BK_FSEED;
  if (t <= S + 1) {
    *k = t - 1;
    return BK_FPROP;
  }
  if (t == S + 2) return BK_VSEED;
  if (t <= 2 * S + 2) {
    *k = 2 * S + 3 - t;
    return BK_VPROP;
  }
  if (t == 2 * S + 3) return BK_TRACE;
  if (t == 2 * S + 4) return BK_GUIDE;
  if (t <= 3 * S + 4) {
    *k = 3 * S + 5 - t;
    return BK_WPROP;
  }
  if (t == 3 * S + 5) return BK_CHAIN;
  return BK_DONE;
}

__device__ __forceinline__ long long batch_now() {
  long long ns;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(ns));
  return ns;
}

__device__ __forceinline__ unsigned long long ld_volatile_u64(const unsigned long long* p) {
  return *(const volatile unsigned long long*)p;
}

// Thread 0: the next published item, or x = 0 when every problem is done or
// the launch gave up.  Slots are handed out in order; a block waits for its
// slot to be published while other blocks make progress, and gives up
// (error 1) when no item has completed anywhere for timeout_ns.
__device__ int4 batch_take(const BatchQueue& q, int n, long long timeout_ns) {
  const unsigned long long it = atomicAdd(q.ctl + 0, 1ull);
  if ((long long)it >= q.cap) {
    atomicCAS(q.ctl + 4, 0ull, 2ull);
    return make_int4(0, 0, 0, 0);
  }
  volatile int* slot = (volatile int*)(q.items + it);
  unsigned long long seen = ld_volatile_u64(q.ctl + 3);
  long long t0 = batch_now();
  for (;;) {
    const int x = slot[0];
    if (x != 0) {
      __threadfence();
      return make_int4(x, slot[1], slot[2], slot[3]);
    }
    if (ld_volatile_u64(q.ctl + 2) >= (unsigned long long)n || ld_volatile_u64(q.ctl + 4) != 0)
      return make_int4(0, 0, 0, 0);
    const unsigned long long p = ld_volatile_u64(q.ctl + 3);
    const long long t = batch_now();
    if (p != seen) {
      seen = p;
      t0 = t;
    } else if (t - t0 > timeout_ns) {
      atomicCAS(q.ctl + 4, 0ull, 1ull);
      return make_int4(0, 0, 0, 0);
    }
    __nanosleep(200);
  }
}

// Tiles of level k's output that can take bits: within reach R (in y and z)
// of the source set's box, and inside the output mask's box when there is
// one.  Returns the count; *t0 / *t1 the tile ranges (ty0, tz0) .. (ty1, tz1).
__device__ __forceinline__ int batch_tile_range(const Dims& d, const TileCfg& tc, int R, const int32_t* xb,
                                                const int32_t* mb, int* ty0, int* ty1, int* tz0, int* tz1) {
  const int bx0 = __ldcg(xb + 0), by0 = __ldcg(xb + 1), bz0 = __ldcg(xb + 2);
  const int bx1 = -__ldcg(xb + 3), by1 = -__ldcg(xb + 4), bz1 = -__ldcg(xb + 5);
  *ty0 = 0;
  *ty1 = -1;
  *tz0 = 0;
  *tz1 = -1;
  if (bx0 > bx1) return 0;
  int ylo = max(0, by0 - R), yhi = min(d.ny - 1, by1 + R);
  int zlo = max(0, bz0 - R), zhi = min(d.nz - 1, bz1 + R);
  if (mb) {
    if (__ldcg(mb + 0) > -__ldcg(mb + 3)) return 0;  // empty output mask
    ylo = max(ylo, __ldcg(mb + 1));
    yhi = min(yhi, -__ldcg(mb + 4));
    zlo = max(zlo, __ldcg(mb + 2));
    zhi = min(zhi, -__ldcg(mb + 5));
  }
  if (ylo > yhi || zlo > zhi) return 0;
  *ty0 = ylo / tc.TY;
  *ty1 = yhi / tc.TY;
  *tz0 = zlo / tc.TZ;
  *tz1 = zhi / tc.TZ;
  return (*ty1 - *ty0 + 1) * (*tz1 - *tz0 + 1);
}

// Block-wide exclusive prefix sum of one int per thread; *total receives the sum.
__device__ int batch_scan(int v, int* warp_sum, int* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  int incl = v;
  for (int o = 1; o < 32; o <<= 1) {
    const int u = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += u;
  }
  __syncthreads();
  if (lane == 31) warp_sum[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    int x = lane < nwarp ? warp_sum[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += u;
    }
    if (lane < nwarp) warp_sum[lane] = x;
  }
  __syncthreads();
  const int excl = (warp > 0 ? warp_sum[warp - 1] : 0) + incl - v;
  *total = warp_sum[nwarp - 1];
  __syncthreads();
  return excl;
}

// Block-wide: moves problem i past its finished stage, publishing the items
// of the next stage that has any (stages without items -- a propagation
// whose source set is empty -- complete at once; their outputs are already
// zero and their boxes empty).  Reaching the end counts the problem done.
__device__ void batch_advance(const BatchProb& P, int i, const BatchQueue& q) {
  __shared__ int warp_sum[32];
  __shared__ int s_stage;
  __shared__ unsigned long long s_base;
  const int S = P.S, W = P.W;
  if (threadIdx.x == 0) s_stage = __ldcg(&q.state[i].x);
  __syncthreads();
  for (int t = s_stage + 1;; ++t) {
    int k = 0;
    const BatchKind kind = batch_kind(S, t, &k);
    if (kind == BK_DONE) {
      if (threadIdx.x == 0) {
        q.state[i] = make_int2(t, 0);
        __threadfence();
        atomicAdd(q.ctl + 2, 1ull);
      }
      return;
    }
    // how many items, and (for the propagation levels) each query's tiles
    int Q = 1;
    const int32_t *xb0 = nullptr, *mb = nullptr;
    long qbs = 0;
    int R = 0;
    TileCfg tc = P.tcs[max(k, 1) - 1];
    if (kind == BK_FPROP) {
      xb0 = P.Fbox + 6 * (k - 1);
      R = P.arm.segf[k - 1].R;
    } else if (kind == BK_VPROP) {
      xb0 = P.Vbox + 6 * k;
      mb = P.Fbox + 6 * (k - 1);
      R = P.arm.seg[k - 1].R;
    } else if (kind == BK_WPROP) {
      Q = W;
      xb0 = P.Vwbox + 6 * k;
      qbs = 6L * (S + 1);
      mb = P.Fbox + 6 * (k - 1);
      R = P.arm.seg[k - 1].R;
    }
    // waypoint levels whose tiling allows it take the queries in pairs
    // (items (tile, pair): the union of both queries' tile ranges)
    const bool pairs = kind == BK_WPROP && tc.pair;
    auto range = [&](int qq, int* ty0, int* ty1, int* tz0, int* tz1) {
      if (!pairs) return batch_tile_range(P.d, tc, R, xb0 + qq * qbs, mb, ty0, ty1, tz0, tz1);
      int a0, a1, b0, b1, c0 = 0, c1 = -1, e0 = 0, e1 = -1;
      const int ca = batch_tile_range(P.d, tc, R, xb0 + 2 * qq * qbs, mb, &a0, &a1, &b0, &b1);
      const int cb = 2 * qq + 1 < W ? batch_tile_range(P.d, tc, R, xb0 + (2 * qq + 1) * qbs, mb, &c0, &c1, &e0, &e1)
                                    : 0;
      if (!ca && !cb) return 0;
      if (!ca) a0 = c0, a1 = c1, b0 = e0, b1 = e1;
      else if (cb) a0 = min(a0, c0), a1 = max(a1, c1), b0 = min(b0, e0), b1 = max(b1, e1);
      *ty0 = a0, *ty1 = a1, *tz0 = b0, *tz1 = b1;
      return (a1 - a0 + 1) * (b1 - b0 + 1);
    };
    if (pairs) Q = (W + 1) / 2;
    int total = 0;
    if (xb0) {
      // one query per thread and pass; items in query order
      for (int q0 = 0; q0 < Q; q0 += blockDim.x) {
        const int qq = q0 + threadIdx.x;
        int ty0, ty1, tz0, tz1, c = 0;
        if (qq < Q) c = range(qq, &ty0, &ty1, &tz0, &tz1);
        int part = 0;
        batch_scan(c, warp_sum, &part);
        total += part;
      }
    } else {
      total = kind == BK_GUIDE ? W : 1;
    }
    if (total == 0) continue;  // nothing to do at this stage
    if (threadIdx.x == 0) {
      q.state[i] = make_int2(t, total);
      __threadfence();
      const unsigned long long base = atomicAdd(q.ctl + 1, (unsigned long long)total);
      s_base = base;
      if ((long long)(base + total) > q.cap) atomicCAS(q.ctl + 4, 0ull, 2ull);
    }
    __syncthreads();
    const unsigned long long base = s_base;
    auto put = [&](long long idx, int a, int b) {
      const unsigned long long at = base + (unsigned long long)idx;
      if ((long long)at >= q.cap) return;
      volatile int* slot = (volatile int*)(q.items + at);
      slot[1] = t;
      slot[2] = a;
      slot[3] = b;
      __threadfence();
      slot[0] = i + 1;
    };
    if (xb0) {
      long long run = 0;
      for (int q0 = 0; q0 < Q; q0 += blockDim.x) {
        const int qq = q0 + threadIdx.x;
        int ty0 = 0, ty1 = -1, tz0 = 0, tz1 = -1, c = 0;
        if (qq < Q) c = range(qq, &ty0, &ty1, &tz0, &tz1);
        int part = 0;
        const int off = batch_scan(c, warp_sum, &part);
        long long n = 0;
        for (int tz = tz0; tz <= tz1; ++tz)
          for (int ty = ty0; ty <= ty1; ++ty, ++n) put(run + off + n, tz * tc.tiles_y + ty, qq);
        run += part;
      }
    } else {
      for (int j = threadIdx.x; j < total; j += blockDim.x) put(j, j, 0);
    }
    return;
  }
}

__device__ void batch_raster(const BatchProb& P, int slab, int32_t* sb) {
  const Dims& d = P.d;
  const int nb = P.n_boxes;
  for (int x = threadIdx.x; x < 6 * nb; x += blockDim.x) sb[x] = __ldg(P.boxes + x);
  __syncthreads();
  const int z0 = slab * kBatchSlab, z1 = min(d.nz, z0 + kBatchSlab);
  const long w0 = (long)z0 * d.ny * d.wx, w1 = (long)z1 * d.ny * d.wx;
  for (long w = w0 + threadIdx.x; w < w1; w += blockDim.x) {
    int wx, y, z;
    word_coords(d, w, &wx, &y, &z);
    uint32_t acc = 0;
    for (int b = 0; b < nb; ++b) {
      const int32_t* B = sb + 6 * b;
      if (y < B[1] || y > B[4] || z < B[2] || z > B[5]) continue;
      const int x0 = max(B[0], 32 * wx), x1 = min(B[3], 32 * wx + 31);
      if (x0 > x1) continue;
      const int lo = x0 - 32 * wx, hi = x1 - 32 * wx;
      const uint32_t upto = hi == 31 ? 0xffffffffu : ((1u << (hi + 1)) - 1u);
      acc |= upto & ~((1u << lo) - 1u);
    }
    P.occ[w] = acc;
  }
}

// Forward seed: every box of the problem starts empty; F_0 = {root} if free.
__device__ void batch_fseed(const BatchProb& P) {
  const int S = P.S, W = P.W;
  const int n_f = 6 * (S + 1), n_w = 6 * (S + 1) * W;
  for (int x = threadIdx.x; x < n_f; x += blockDim.x) {
    P.Fbox[x] = 0x7f7f7f7f;
    P.Vbox[x] = 0x7f7f7f7f;
  }
  for (int x = threadIdx.x; x < n_w; x += blockDim.x) P.Vwbox[x] = 0x7f7f7f7f;
  __syncthreads();
  if (threadIdx.x == 0) {
    const Dims& d = P.d;
    const long r = lin(d, P.root[0], P.root[1], P.root[2]);
    if (!((__ldg(P.occ + (r >> 5)) >> (r & 31)) & 1u)) {
      P.F[r >> 5] = 1u << (r & 31);
      box_point(P.Fbox, P.root[0], P.root[1], P.root[2]);
    }
  }
}

// Reach seed: V_S = {target} & F_S.
__device__ void batch_vseed(const BatchProb& P) {
  if (threadIdx.x != 0) return;
  const Dims& d = P.d;
  const int S = P.S;
  const long t = lin(d, P.target[0], P.target[1], P.target[2]);
  if ((__ldg(P.F + (long)S * d.nw + (t >> 5)) >> (t & 31)) & 1u) {
    P.V[(long)S * d.nw + (t >> 5)] = 1u << (t & 31);
    box_point(P.Vbox + 6 * S, P.target[0], P.target[1], P.target[2]);
  }
}

__device__ void batch_chain(const BatchProb& P, const BatchRules& r, ChainShared& sh, int* rad, uint32_t* so) {
  const int S = P.S, W = P.W;
  const int pose_ints = 3 * (S + 1);
  // mode 0 starts from the reach pose at the last waypoint
  for (int x = threadIdx.x; x < pose_ints; x += blockDim.x) P.poses[(long)(W - 1) * pose_ints + x] = P.reach[x];
  __syncthreads();
  ChainArgs a;
  a.P = 1;
  a.W = W;
  a.c = 0;
  a.mode = 0;
  a.delta = r.delta;
  a.max_relax = r.max_relax;
  a.found = P.found;
  a.Vw = P.Vw;
  a.eps_used = P.eps;
  a.poses = P.poses;
  a.relax = P.relax;
  a.status = P.status;
  a.scratch = P.chain;
  a.relaxed_eps_base = r.eps2;
  a.c_arr = nullptr;
  a.per_joint = false;
  a.rad[0] = -1;
  for (int k = 1; k <= IK_MAX_SEG; ++k) a.rad[k] = r.delta;
  a.vbox = P.Vwbox;
  a.counters = nullptr;
  smooth_chain_block(P.d, P.arm, a, 0, sh, rad, so);
  __syncthreads();
  // the packed outputs
  for (int x = threadIdx.x; x < pose_ints; x += blockDim.x) P.o_reach[x] = P.reach[x];
  for (long x = threadIdx.x; x < (long)W * pose_ints; x += blockDim.x) P.o_poses[x] = P.poses[x];
  for (int x = threadIdx.x; x < 2 * W; x += blockDim.x) P.o_relax[x] = P.relax[x];
  if (threadIdx.x == 0) {
    *P.o_found = *P.found;
    *P.o_status = *P.status;
    *P.o_rc = IK_OK;
  }
}

__global__ void __launch_bounds__(kBatchThreads, 1) k_batch_persistent(const BatchProb* __restrict__ probs, int n,
                                                                       BatchQueue q, BatchRules r,
                                                                       long long timeout_ns) {
  extern __shared__ uint32_t dyn[];
  __shared__ ChainShared csh;
  __shared__ int crad[IK_MAX_SEG + 1];
  __shared__ int4 s_item;
  __shared__ int s_last;
  for (;;) {
    if (threadIdx.x == 0) s_item = batch_take(q, n, timeout_ns);
    __syncthreads();
    const int4 it = s_item;
    if (it.x <= 0) break;
    const int i = it.x - 1;
    const BatchProb& P = probs[i];
    const Dims d = P.d;
    const int S = P.S;
    int k = 0;
    const BatchKind kind = batch_kind(S, it.y, &k);
    switch (kind) {
      case BK_RASTER:
        batch_raster(P, it.z, (int32_t*)dyn);
        break;
      case BK_FSEED:
        batch_fseed(P);
        break;
      case BK_FPROP: {
        const SegDev seg = P.arm.segf[k - 1];
        const TileCfg tc = P.tcs[k - 1];
        propagate_tile_body<false, true, true>(d, seg, tc, P.F + (long)(k - 1) * d.nw, 0, nullptr, 0, P.occ,
                                              P.F + (long)k * d.nw, 0, P.Fbox + 6 * (k - 1), P.Fbox + 6 * k,
                                              0, nullptr, 0, it.z);
        break;
      }
      case BK_VSEED:
        batch_vseed(P);
        break;
      case BK_VPROP: {
        const SegDev seg = P.arm.seg[k - 1];
        const TileCfg tc = P.tcs[k - 1];
        propagate_tile_body<false, true, true>(d, seg, tc, P.V + (long)k * d.nw, 0, P.F + (long)(k - 1) * d.nw,
                                              0, P.occ, P.V + (long)(k - 1) * d.nw, 0, P.Vbox + 6 * k,
                                              P.Vbox + 6 * (k - 1), 0, nullptr, 0, it.z);
        break;
      }
      case BK_TRACE:
        traceback_block(d, P.arm, P.root[0], P.root[1], P.root[2], P.V, nullptr, P.reach, P.found);
        break;
      case BK_GUIDE: {
        GuideArm ga;
        ga.S = S;
        for (int x = 0; x < S; ++x) ga.len[x] = P.arm.len[x];
        guide_targets_block(d, P.arm, ga, P.occ, P.F + (long)S * d.nw, P.reach, P.found, P.W, r.eps2,
                            r.eps2_max, P.g, P.eps, P.Vw, P.Vwbox, nullptr, nullptr, 0, it.z);
        break;
      }
      case BK_WPROP: {
        const SegDev seg = P.arm.seg[k - 1];
        const TileCfg tc = P.tcs[k - 1];
        const long qs = (long)(S + 1) * d.nw;
        if (tc.pair)  // it.w: a pair of waypoint queries sharing the supercover walks
          propagate_pair_body<false, false, true, true>(d, seg, tc, P.Vw + (long)k * d.nw, qs,
                                                        P.F + (long)(k - 1) * d.nw, P.occ,
                                                        P.Vw + (long)(k - 1) * d.nw, qs, P.W, P.Vwbox + 6 * k,
                                                        P.Vwbox + 6 * (k - 1), 6L * (S + 1), nullptr, it.z, it.w);
        else
          propagate_tile_body<false, true, true>(d, seg, tc, P.Vw + (long)k * d.nw, qs, P.F + (long)(k - 1) * d.nw,
                                                0, P.occ, P.Vw + (long)(k - 1) * d.nw, qs, P.Vwbox + 6 * k,
                                                P.Vwbox + 6 * (k - 1), 6L * (S + 1), nullptr, it.w, it.z);
        break;
      }
      case BK_CHAIN:
        batch_chain(P, r, csh, crad, dyn);
        break;
      default:
        break;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();  // this item's writes before its completion is counted
      const int left = atomicSub(&q.state[i].y, 1) - 1;
      atomicAdd(q.ctl + 3, 1ull);
      s_last = left == 0;
      if (left == 0) __threadfence();  // and every other item of the stage before the next one
    }
    __syncthreads();
    if (s_last) batch_advance(P, i, q);
    __syncthreads();
  }
}

size_t batch_chain_smem_bytes() { return (size_t)(kChainOccWords + kChainSrcWords) * sizeof(uint32_t); }

size_t batch_smem_limit() {
  int dev = 0, optin = 0;
  cudaFuncAttributes fa;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
      cudaFuncGetAttributes(&fa, (const void*)k_batch_persistent) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return (size_t)optin > fa.sharedSizeBytes ? (size_t)optin - fa.sharedSizeBytes : 0;
}

// The attribute belongs to the kernel, not to an engine: every engine of the
// process shares it, so it only ever grows (per device, under a lock), and
// a launch never finds it lowered by another engine.
cudaError_t batch_set_smem(size_t bytes) {
  static std::mutex mu;
  static size_t set_bytes[64] = {0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(mu);
  if (bytes <= set_bytes[dev]) return cudaSuccess;
  e = cudaFuncSetAttribute((const void*)k_batch_persistent, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) set_bytes[dev] = bytes;
  return e;
}

cudaError_t launch_batch_persistent(const BatchProb* probs, int n, const BatchQueue& q, const BatchRules& r,
                                    int blocks, size_t smem, long long timeout_ns, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_batch_persistent<<<blocks, kBatchThreads, smem, st>>>(probs, n, q, r, timeout_ns);
  return cudaGetLastError();
}
