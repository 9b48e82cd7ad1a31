// sm_103a kernels of the lattice gap map-seeking IK hot path.
//
// Voxel sets are x-packed bitsets: bit b of word (z*ny + y)*wx + w is voxel
// (32w + b, y, z).  A set shifted by an offset (dx, dy, dz) is read 32 voxels
// at a time with one or two word loads and a funnel shift; voxels outside the
// grid read as 0.  Everything here is exact boolean arithmetic.

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>
#include <type_traits>

#include "ik_internal.h"

namespace ikb {

// ------------------------------------------------------------------ helpers

__device__ __forceinline__ void word_coords(const Dims& d, long w, int* wx, int* y, int* z) {
  *wx = (int)(w % d.wx);
  long r = w / d.wx;
  *y = (int)(r % d.ny);
  *z = (int)(r / d.ny);
}

// Bits of voxels (32*wx + b + dx, y + dy, z + dz), b = 0..31, of set s.
__device__ __forceinline__ uint32_t ld_shifted(const uint32_t* __restrict__ s, const Dims& d, int wx,
                                               int y, int z, int dx, int dy, int dz) {
  const int yy = y + dy, zz = z + dz;
  if ((unsigned)yy >= (unsigned)d.ny || (unsigned)zz >= (unsigned)d.nz) return 0u;
  const uint32_t* row = s + ((long)zz * d.ny + yy) * d.wx;
  const int w0 = wx + (dx >> 5);
  const int sh = dx & 31;
  const uint32_t lo = ((unsigned)w0 < (unsigned)d.wx) ? __ldg(row + w0) : 0u;
  if (sh == 0) return lo;
  const uint32_t hi = ((unsigned)(w0 + 1) < (unsigned)d.wx) ? __ldg(row + w0 + 1) : 0u;
  return __funnelshift_r(lo, hi, sh);
}

__device__ __forceinline__ bool inside(const Dims& d, int x, int y, int z) {
  return (unsigned)x < (unsigned)d.nx && (unsigned)y < (unsigned)d.ny && (unsigned)z < (unsigned)d.nz;
}

__device__ __forceinline__ long lin(const Dims& d, int x, int y, int z) {
  return ((long)z * d.ny + y) * d.nx + x;
}

__device__ __forceinline__ bool test_bit(const uint32_t* s, long i) {
  return (__ldg(s + (i >> 5)) >> (i & 31)) & 1u;
}

// Free bits of the segments from the 32 voxels of word (wx, y, z) along
// offset e of the shell: the stored edge-mask word when the grid keeps edge
// masks, else the supercover of e walked against the occupancy.
__device__ __forceinline__ uint32_t edge_word(const Dims& d, const SegDev& sg, int e, long w, int wx,
                                              int y, int z) {
  if (sg.mask) return __ldg(sg.mask + (long)e * sg.mbox.words() + sg.mbox.index(wx, y, z));
  const int s1 = __ldg(sg.sc_start + e + 1);
  uint32_t blocked = 0;
  int i = __ldg(sg.sc_start + e);
  // four independent voxel reads per pass; the all-blocked exit is checked
  // once per pass so that the reads do not wait on each other
  for (; i + 4 <= s1 && blocked != 0xffffffffu; i += 4) {
    uint32_t b[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int32_t v = __ldg(sg.sc + i + u);
      b[u] = ld_shifted(sg.occ, d, wx, y, z, unpack_x(v), unpack_y(v), unpack_z(v));
    }
    blocked |= b[0] | b[1] | b[2] | b[3];
  }
  for (; i < s1; ++i) {
    const int32_t v = __ldg(sg.sc + i);
    blocked |= ld_shifted(sg.occ, d, wx, y, z, unpack_x(v), unpack_y(v), unpack_z(v));
  }
  return ~blocked;
}

// The same free bits from an occupancy halo staged in shared memory with the
// layout of the tiled kernels: base is the lane's own word in the halo and
// sctab holds each supercover voxel's shared-memory delta and x shift.
__device__ __forceinline__ uint32_t edge_word_tile(const SegDev& sg, int e, const uint32_t* so,
                                                   int base) {
  const int s1 = __ldg(sg.sc_start + e + 1);
  uint32_t blocked = 0;
  int i = __ldg(sg.sc_start + e);
  for (; i + 4 <= s1 && blocked != 0xffffffffu; i += 4) {
    uint32_t b[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int32_t t = __ldg(sg.sctab + i + u);
      const int a = base + (t >> 5);
      b[u] = __funnelshift_r(so[a], so[a + 1], t);  // shift taken mod 32
    }
    blocked |= b[0] | b[1] | b[2] | b[3];
  }
  for (; i < s1; ++i) {
    const int32_t t = __ldg(sg.sctab + i);
    const int a = base + (t >> 5);
    blocked |= __funnelshift_r(so[a], so[a + 1], t);
  }
  return ~blocked;
}

// The segment from voxel p (linear index pi) along offset e: free?
__device__ __forceinline__ bool edge_bit(const Dims& d, const SegDev& sg, int e, long pi) {
  const long w = pi >> 5;
  const int wx = (int)(w % d.wx), y = (int)((w / d.wx) % d.ny), z = (int)(w / ((long)d.wx * d.ny));
  return (edge_word(d, sg, e, w, wx, y, z) >> (pi & 31)) & 1u;
}

static inline int grid_for(long n, int block) { return (int)((n + block - 1) / block); }

// ----------------------------------------------------------- rasterise boxes

// One thread per occupancy word: OR of the x-runs of every box that covers
// the word's row.  Boxes are staged through shared memory in chunks.
constexpr int kBoxChunk = 512;

__global__ void k_rasterize(Dims d, const int32_t* __restrict__ boxes, int nb, uint32_t* occ) {
  __shared__ int32_t sb[kBoxChunk * 6];
  const long w = blockIdx.x * (long)blockDim.x + threadIdx.x;
  int wx = 0, y = 0, z = 0;
  if (w < d.nw) word_coords(d, w, &wx, &y, &z);
  uint32_t acc = 0;
  for (int base = 0; base < nb; base += kBoxChunk) {
    const int cnt = min(kBoxChunk, nb - base);
    __syncthreads();
    for (int i = threadIdx.x; i < cnt * 6; i += blockDim.x) sb[i] = boxes[(long)base * 6 + i];
    __syncthreads();
    if (w < d.nw) {
      for (int b = 0; b < cnt; ++b) {
        const int32_t* B = sb + 6 * b;
        if (y < B[1] || y > B[4] || z < B[2] || z > B[5]) continue;
        const int x0 = max(B[0], 32 * wx), x1 = min(B[3], 32 * wx + 31);
        if (x0 > x1) continue;
        const int lo = x0 - 32 * wx, hi = x1 - 32 * wx;
        const uint32_t upto = hi == 31 ? 0xffffffffu : ((1u << (hi + 1)) - 1u);
        acc |= upto & ~((1u << lo) - 1u);
      }
    }
  }
  if (w < d.nw) occ[w] = acc;
}

// Obstacle dilation by the ball |v|^2 <= r2: dst[p] = OR over the ball of
// src[p + v], one thread per word (the ball is symmetric, so this gather is
// the dilation); each (dz, dy) row of the ball is one run of dx.
__global__ void k_dilate(Dims d, const uint32_t* __restrict__ src, int r2, uint32_t* __restrict__ dst) {
  const long w = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (w >= d.nw) return;
  int wx, y, z;
  word_coords(d, w, &wx, &y, &z);
  int r = 0;
  while ((r + 1) * (r + 1) <= r2) ++r;
  uint32_t acc = 0;
  for (int dz = -r; dz <= r && acc != 0xffffffffu; ++dz) {
    for (int dy = -r; dy <= r; ++dy) {
      const int rem = r2 - dz * dz - dy * dy;
      if (rem < 0) continue;
      int b = 0;
      while ((b + 1) * (b + 1) <= rem) ++b;
      for (int dx = -b; dx <= b; ++dx) acc |= ld_shifted(src, d, wx, y, z, dx, dy, dz);
    }
  }
  dst[w] = acc;
}

cudaError_t launch_dilate(const Dims& d, const uint32_t* src, int r2, uint32_t* dst, cudaStream_t st) {
  k_dilate<<<grid_for(d.nw, 256), 256, 0, st>>>(d, src, r2, dst);
  return cudaGetLastError();
}

cudaError_t launch_rasterize(const Dims& d, const int32_t* boxes, int n_boxes, uint32_t* occ,
                             cudaStream_t st) {
  k_rasterize<<<grid_for(d.nw, 256), 256, 0, st>>>(d, boxes, n_boxes, occ);
  return cudaGetLastError();
}

// ----------------------------------------------- edge masks (per-offset M_e)

// M_e[p] = AND over v in SC(0, e) of free(p + v): the segment p -> p + e is
// obstacle-free.  One thread per (offset, word); the offset's supercover list
// is uniform across the block (blockIdx.y = offset).
__global__ void k_edge_masks(Dims d, MaskBox b, const uint32_t* __restrict__ occ,
                             const int32_t* __restrict__ sc_start, const int32_t* __restrict__ sc,
                             int n_off, uint32_t* __restrict__ mask) {
  const long nb = b.words();
  for (int e = blockIdx.y; e < n_off; e += gridDim.y) {
    const int s0 = __ldg(sc_start + e), s1 = __ldg(sc_start + e + 1);
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < nb; t += (long)gridDim.x * blockDim.x) {
      const int wx = b.wx0 + (int)(t % b.nwx()), y = b.y0 + (int)((t / b.nwx()) % b.nyy());
      const int z = b.z0 + (int)(t / ((long)b.nwx() * b.nyy()));
      uint32_t blocked = 0;
      for (int i = s0; i < s1 && blocked != 0xffffffffu; ++i) {
        const int32_t v = __ldg(sc + i);
        blocked |= ld_shifted(occ, d, wx, y, z, unpack_x(v), unpack_y(v), unpack_z(v));
      }
      mask[(long)e * nb + t] = ~blocked;
    }
  }
}

// Shared-memory form: a block covers one output tile (TileCfg) and a chunk
// of kMaskChunk offsets.  The occupancy halo of the tile (reach R, zero
// outside the grid, where a segment cannot end anyway) is staged once and
// reused for every offset of the chunk; each supercover voxel is then two
// shared loads and a funnel shift at a precomputed delta.
constexpr int kMaskChunk = 64;

__global__ void __launch_bounds__(256) k_edge_masks_tile(Dims d, TileCfg tc, MaskBox b, int tiles_y,
                                                         int R, int n_off,
                                                         const uint32_t* __restrict__ occ,
                                                         const int32_t* __restrict__ sc_start,
                                                         const int32_t* __restrict__ sctab,
                                                         uint32_t* __restrict__ mask) {
  extern __shared__ uint32_t so[];
  // tiles of the mask box (y and z); a tile still spans every word of its rows
  const int y0 = b.y0 + (blockIdx.x % tiles_y) * tc.TY, z0 = b.z0 + (blockIdx.x / tiles_y) * tc.TZ;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int RY = tc.TY + 2 * R, RZ = tc.TZ + 2 * R, P = tc.P;
  const int n_rows = RZ * RY;
  if ((d.wx & 3) == 0) {
    // rows of 16-byte multiples: one thread per staged row, 128-bit loads
    // (one per four words), the two pad words zero
    for (int r = threadIdx.x; r < n_rows; r += blockDim.x) {
      const int sy = y0 - R + r % RY, sz = z0 - R + r / RY;
      uint32_t* dst = so + r * P;
      dst[0] = 0u;
      dst[d.wx + 1] = 0u;
      if (sy >= 0 && sy < d.ny && sz >= 0 && sz < d.nz) {
        const uint4* src = reinterpret_cast<const uint4*>(occ + ((long)sz * d.ny + sy) * d.wx);
        for (int q = 0; q < (d.wx >> 2); ++q) {
          const uint4 v = __ldg(src + q);
          dst[1 + 4 * q] = v.x;
          dst[2 + 4 * q] = v.y;
          dst[3 + 4 * q] = v.z;
          dst[4 + 4 * q] = v.w;
        }
      } else {
        for (int c = 1; c <= d.wx; ++c) dst[c] = 0u;
      }
    }
  } else {
    const int per_pass = 32 / P;
    const int sub = lane / P, c = lane % P, sw = c - 1;
    if (sub < per_pass) {
      for (int r = warp * per_pass + sub; r < n_rows; r += 8 * per_pass) {
        const int sy = y0 - R + r % RY, sz = z0 - R + r / RY;
        uint32_t v = 0u;
        if (sw >= 0 && sw < d.wx && sy >= 0 && sy < d.ny && sz >= 0 && sz < d.nz)
          v = __ldg(occ + ((long)sz * d.ny + sy) * d.wx + sw);
        so[r * P + c] = v;
      }
    }
  }
  __syncthreads();
  const int z = z0 + warp, wx = lane % d.wx, y = y0 + lane / d.wx;
  if (warp >= tc.TZ || lane >= tc.lanes || y > b.y1 || z > b.z1 || wx < b.wx0 || wx > b.wx1) return;
  const long w = b.index(wx, y, z), nb = b.words();
  const int base = ((z - z0 + R) * RY + (y - y0 + R)) * P + (wx + 1);
  const int e_end = min(n_off, (int)(blockIdx.y + 1) * kMaskChunk);
  for (int e = blockIdx.y * kMaskChunk; e < e_end; ++e) {
    const int s1 = __ldg(sc_start + e + 1);
    uint32_t blocked = 0;
    int i = __ldg(sc_start + e);
    for (; i + 4 <= s1; i += 4) {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int32_t t = __ldg(sctab + i + u);
        const int a = base + (t >> 5);
        blocked |= __funnelshift_r(so[a], so[a + 1], t & 31);
      }
    }
    for (; i < s1; ++i) {
      const int32_t t = __ldg(sctab + i);
      const int a = base + (t >> 5);
      blocked |= __funnelshift_r(so[a], so[a + 1], t & 31);
    }
    mask[(long)e * nb + w] = ~blocked;
  }
}

// The same edge masks with the occupancy brick of a tile (its halo of reach
// R in y and z, words -4 .. BX - 5 in x) copied into shared memory by one
// TMA tensor load (cp.async.bulk.tensor, completion on an mbarrier) instead
// of per-thread loads.  The copy starts at word -4 because a tiled copy's
// innermost coordinate must be a multiple of 16 bytes; the words outside
// the grid arrive as zeros (the tensor map's out-of-bounds fill), so word
// w of a row sits at column w + 4 of a BX-word staged row.  sctab holds the
// supercover deltas for that pitch.  The wait is bounded: if the copy has
// not completed after kTmaWaitNs, the block stages the brick with plain
// loads instead (the same values, so a late copy changes nothing) and
// counts the event in *slow.
constexpr long long kTmaWaitNs = 200LL * 1000 * 1000;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__global__ void __launch_bounds__(256) k_edge_masks_tma(const __grid_constant__ CUtensorMap tmap, Dims d,
                                                        TileCfg tc, MaskBox b, int tiles_y, int R, int n_off,
                                                        int BX, const uint32_t* __restrict__ occ,
                                                        const int32_t* __restrict__ sc_start,
                                                        const int32_t* __restrict__ sctab,
                                                        uint32_t* __restrict__ mask, int* slow) {
  extern __shared__ __align__(128) uint32_t so_raw[];
  __shared__ __align__(8) unsigned long long bar;
  // the copy's destination: 128-byte aligned
  uint32_t* so = (uint32_t*)(((uintptr_t)so_raw + 127) & ~(uintptr_t)127);
  const int y0 = b.y0 + (blockIdx.x % tiles_y) * tc.TY, z0 = b.z0 + (blockIdx.x / tiles_y) * tc.TZ;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int RY = tc.TY + 2 * R, RZ = tc.TZ + 2 * R;
  const uint32_t bytes = (uint32_t)BX * RY * RZ * 4u;
  const uint32_t bar_a = smem_u32(&bar);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_a) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar_a), "r"(bytes) : "memory");
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(smem_u32(so)),
        "l"((unsigned long long)&tmap), "r"(-4), "r"(y0 - R), "r"(z0 - R), "r"(bar_a)
        : "memory");
  }
  __syncthreads();  // the barrier is initialised before anyone waits on it
  uint32_t done = 0;
  long long t0;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  for (;;) {
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar_a)
        : "memory");
    if (done) break;
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    if (t - t0 > kTmaWaitNs) break;
  }
  if (!__syncthreads_and(done)) {
    // fall back to plain loads of the same brick
    if (threadIdx.x == 0) atomicAdd(slow, 1);
    const int n = RZ * RY * BX;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const int c = i % BX, r = (i / BX) % RY, zz = i / (BX * RY);
      const int sw = c - 4, sy = y0 - R + r, sz = z0 - R + zz;
      uint32_t v = 0u;
      if (sw >= 0 && sw < d.wx && sy >= 0 && sy < d.ny && sz >= 0 && sz < d.nz)
        v = __ldg(occ + ((long)sz * d.ny + sy) * d.wx + sw);
      so[i] = v;
    }
    __syncthreads();
  }
  const int z = z0 + warp, wx = lane % d.wx, y = y0 + lane / d.wx;
  if (warp >= tc.TZ || lane >= tc.lanes || y > b.y1 || z > b.z1 || wx < b.wx0 || wx > b.wx1) return;
  const long w = b.index(wx, y, z), nb = b.words();
  const int base = ((z - z0 + R) * RY + (y - y0 + R)) * BX + (wx + 4);
  const int e_end = min(n_off, (int)(blockIdx.y + 1) * kMaskChunk);
  for (int e = blockIdx.y * kMaskChunk; e < e_end; ++e) {
    const int s1 = __ldg(sc_start + e + 1);
    uint32_t blocked = 0;
    int i = __ldg(sc_start + e);
    for (; i + 4 <= s1; i += 4) {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int32_t t = __ldg(sctab + i + u);
        const int a = base + (t >> 5);
        blocked |= __funnelshift_r(so[a], so[a + 1], t & 31);
      }
    }
    for (; i < s1; ++i) {
      const int32_t t = __ldg(sctab + i);
      const int a = base + (t >> 5);
      blocked |= __funnelshift_r(so[a], so[a + 1], t & 31);
    }
    mask[(long)e * nb + w] = ~blocked;
  }
}

size_t tma_mask_smem_bytes(const TileCfg& tc, int R, int BX) {
  if (BX <= 0 || R > 31) return 0;
  const size_t bytes = (size_t)BX * (tc.TY + 2 * R) * (tc.TZ + 2 * R) * 4 + 128;
  return bytes <= (size_t)kTileOccSmemMax ? bytes : 0;
}

int tma_mask_pitch(const Dims& d) {
  // rows must be a multiple of 16 bytes apart for a tensor map
  if ((d.wx * 4) % 16 != 0) return 0;
  return (d.wx + 5 + 3) / 4 * 4;
}

cudaError_t launch_edge_masks_tma(const Dims& d, const TileCfg& tc, const void* tmap, const uint32_t* occ,
                                  const ShellDev& s, const MaskBox& b, uint32_t* mask, int* slow,
                                  cudaStream_t st) {
  const int n = (int)s.host.off.size();
  if (n == 0 || b.words() <= 0) return cudaSuccess;
  const int BX = tma_mask_pitch(d);
  const size_t smem = tma_mask_smem_bytes(tc, s.reach, BX);
  if (!smem || !s.d_sctab_tma) return cudaErrorInvalidValue;
  const int tiles_y = (b.nyy() + tc.TY - 1) / tc.TY, tiles_z = (b.z1 - b.z0 + tc.TZ) / tc.TZ;
  dim3 grid(tiles_y * tiles_z, (n + kMaskChunk - 1) / kMaskChunk);
  k_edge_masks_tma<<<grid, 256, smem, st>>>(*(const CUtensorMap*)tmap, d, tc, b, tiles_y, s.reach, n, BX, occ,
                                            s.d_sc_start, s.d_sctab_tma, mask, slow);
  return cudaGetLastError();
}

cudaError_t launch_edge_masks_rows(const Dims& d, const TileCfg& tc, const uint32_t* occ, const ShellDev& s,
                                   const MaskBox& b, uint32_t* mask, cudaStream_t st, bool* done);

cudaError_t launch_edge_masks(const Dims& d, const TileCfg& tc, const uint32_t* occ, const ShellDev& s,
                              const MaskBox& b, uint32_t* mask, cudaStream_t st) {
  const int n = (int)s.host.off.size();
  if (n == 0 || b.words() <= 0) return cudaSuccess;
  {
    bool done = false;
    const cudaError_t e = launch_edge_masks_rows(d, tc, occ, s, b, mask, st, &done);
    if (done || e != cudaSuccess) return e;
  }
  const size_t smem = tile_smem_bytes(tc, s.reach);
  if (smem > 0 && s.d_sctab) {
    const int tiles_y = (b.nyy() + tc.TY - 1) / tc.TY, tiles_z = (b.z1 - b.z0 + tc.TZ) / tc.TZ;
    dim3 grid(tiles_y * tiles_z, (n + kMaskChunk - 1) / kMaskChunk);
    k_edge_masks_tile<<<grid, 256, smem, st>>>(d, tc, b, tiles_y, s.reach, n, occ, s.d_sc_start,
                                               s.d_sctab, mask);
    return cudaGetLastError();
  }
  const int block = 256;
  const int gx = max(1, min(grid_for(b.words(), block), 64));
  dim3 grid(gx, min(n, 65535));
  k_edge_masks<<<grid, block, 0, st>>>(d, b, occ, s.d_sc_start, s.d_sc, n, mask);
  return cudaGetLastError();
}

// ------------------------------------------------------- one propagation D_k

// Warp-level accumulation of the word box of the lanes whose output word is
// non-empty: one atomicMin per component per warp.  Every lane still active
// in the warp must call it.
__device__ __forceinline__ void box_accumulate(int32_t* box, bool nz, int wx, int y, int z) {
  const unsigned act = __activemask();
  if (!__ballot_sync(act, nz)) return;
  const int big = 0x7fffffff;
  const int v0 = __reduce_min_sync(act, nz ? wx : big);
  const int v1 = __reduce_min_sync(act, nz ? y : big);
  const int v2 = __reduce_min_sync(act, nz ? z : big);
  const int v3 = __reduce_min_sync(act, nz ? -wx : big);
  const int v4 = __reduce_min_sync(act, nz ? -y : big);
  const int v5 = __reduce_min_sync(act, nz ? -z : big);
  if ((threadIdx.x & 31) == __ffs(act) - 1) {
    atomicMin(box + 0, v0);
    atomicMin(box + 1, v1);
    atomicMin(box + 2, v2);
    atomicMin(box + 3, v3);
    atomicMin(box + 4, v4);
    atomicMin(box + 5, v5);
  }
}

// out[p] = mask[p] & OR_e X[p + e] & M_e[p] over the shell of segment k.
// Gather form of the scatter "every p reachable from X by a valid segment":
// the shell is symmetric and SC(p, p+e) = p + SC(0, e).
//
// Only offsets whose source voxels can fall inside the word box of X are
// visited.  The walk is warp-uniform: a warp covers 32 consecutive output
// words, takes the union of its lanes' z and y ranges, and for each dz walks
// the one contiguous run of the (z, y, x)-ordered shell table whose dy lies
// in that union; each lane predicates on its own box test.  A lane's edge
// mask word is read only when its shifted input could add new bits, and the
// warp leaves a dz early once every lane holds every free voxel its mask
// allows.
template <bool kCount>
__global__ void __launch_bounds__(256) k_propagate(Dims d, SegDev seg, const uint32_t* __restrict__ X,
                                                   long xs, const uint32_t* __restrict__ mask, long ms,
                                                   const uint32_t* __restrict__ occ,
                                                   uint32_t* __restrict__ out, long os,
                                                   const int32_t* __restrict__ xbox,
                                                   int32_t* __restrict__ obox, long bs,
                                                   unsigned long long* __restrict__ counters) {
  constexpr unsigned kFull = 0xffffffffu;
  const int q = blockIdx.y;
  const long w = blockIdx.x * (long)blockDim.x + threadIdx.x;
  const bool valid = w < d.nw;
  const uint32_t* Xq = X + q * xs;
  const int32_t* xb = xbox + q * bs;
  const int bx0 = __ldg(xb + 0), by0 = __ldg(xb + 1), bz0 = __ldg(xb + 2);
  const int bx1 = -__ldg(xb + 3), by1 = -__ldg(xb + 4), bz1 = -__ldg(xb + 5);
  int wx = 0, y = 0, z = 0;
  uint32_t m = 0;
  if (valid) {
    word_coords(d, w, &wx, &y, &z);
    m = (mask ? __ldg(mask + q * ms + w) : 0xffffffffu) & ~__ldg(occ + w);
  }
  uint32_t acc = 0;
  unsigned long long visited = 0, nonzero = 0, mloads = 0;
  if (bx0 <= bx1 && __any_sync(kFull, m != 0)) {
    const int R = seg.R, side = 2 * R + 1;
    const int big = 0x7fffffff;
    const int zlo = __reduce_min_sync(kFull, m ? z : big), zhi = -__reduce_min_sync(kFull, m ? -z : big);
    const int ylo = __reduce_min_sync(kFull, m ? y : big), yhi = -__reduce_min_sync(kFull, m ? -y : big);
    const int ez0 = max(bz0 - zhi, -R), ez1 = min(bz1 - zlo, R);
    const int ey0 = max(by0 - yhi, -R), ey1 = min(by1 - ylo, R);
    const int exlo = 32 * (bx0 - wx) - 31, exhi = 32 * (bx1 - wx) + 31;
    bool live = m != 0;
    for (int ez = ez0; ez <= ez1 && ey0 <= ey1; ++ez) {
      const int sz = z + ez;
      const bool zok = live && sz >= bz0 && sz <= bz1;
      if (!__any_sync(kFull, zok)) continue;
      const int32_t* rowp = seg.rows + (ez + R) * side + R;
      const int e1 = __ldg(rowp + ey1 + 1);
      for (int e = __ldg(rowp + ey0); e < e1; ++e) {
        const int32_t o = __ldg(seg.off + e);
        const int ex = unpack_x(o), ey = unpack_y(o);
        const int sy = y + ey;
        const bool ok = zok && sy >= by0 && sy <= by1 && ex >= exlo && ex <= exhi;
        if (ok) {
          const uint32_t x = ld_shifted(Xq, d, wx, y, z, ex, ey, ez);
          if (kCount) {
            ++visited;
            nonzero += x != 0;
          }
          if (x & m & ~acc) {
            if (kCount) ++mloads;
            acc |= x & edge_word(d, seg, e, w, wx, y, z);
          }
        }
      }
      live = live && (acc & m) != m;
      if (!__any_sync(kFull, live)) break;
    }
  }
  acc &= m;
  if (valid) out[q * os + w] = acc;
  box_accumulate(obox + q * bs, acc != 0, wx, y, z);
  if (kCount && valid) {
    atomicAdd(counters + 0, visited);
    atomicAdd(counters + 1, nonzero);
    atomicAdd(counters + 2, mloads);
    atomicAdd(counters + 3, (unsigned long long)(m != 0));
  }
}

// Shared-memory form of the same propagation.  The block's output tile is
// all wx words of TY rows in TZ slices; its source halo (reach R in y and z,
// one word in x) is copied from X into shared memory once, with everything
// outside the word box of X (and outside the grid) left zero, so the offset
// walk reads two shared words per offset with no bounds test: the per-offset
// address delta and funnel shift come from the precomputed table tab.  The
// walk visits, per warp (one z slice), the dz range that can reach the box
// of X and, per dz, the one contiguous run of offsets whose dy can reach it
// from any of the warp's rows.
// Slices of a staged halo: TZ + 2R with TZ <= 16 and R <= 31 (the tiled
// kernels' limits).
constexpr int kMaxSlices = 16 + 2 * 31;

// Loads of sets that a persistent launch writes while it runs (kCoh): the
// L2-coherent path instead of the read-only one.
template <bool kCoh>
__device__ __forceinline__ int32_t ld_box(const int32_t* p) {
  return kCoh ? __ldcg(p) : __ldg(p);
}

// The block has blockDim.x / 32 warps (8 for the grid API's kernels, 16 for
// the persistent batch kernel); warp i computes slice z0 + i of the tile
// (warps at or beyond tc.TZ only stage).
template <bool kCount, bool kOcc, bool kCoh = false>
__device__ __forceinline__ void propagate_tile_body(const Dims& d, const SegDev& seg, const TileCfg& tc,
                                                    const uint32_t* __restrict__ X, long xs,
                                                    const uint32_t* __restrict__ mask, long ms,
                                                    const uint32_t* __restrict__ occ,
                                                    uint32_t* __restrict__ out, long os,
                                                    const int32_t* __restrict__ xbox,
                                                    int32_t* __restrict__ obox, long bs,
                                                    unsigned long long* __restrict__ counters, int q,
                                                    int tile) {
  extern __shared__ uint32_t sx[];
  // per staged slice: the rows holding a non-zero source word
  __shared__ int s_ymin[kMaxSlices], s_ymax[kMaxSlices];
  constexpr unsigned kFull = 0xffffffffu;
  const int y0 = (tile % tc.tiles_y) * tc.TY, z0 = (tile / tc.tiles_y) * tc.TZ;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int R = seg.R, RY = tc.TY + 2 * R, P = tc.P;
  const int z = z0 + warp, wx = lane % d.wx, y = y0 + lane / d.wx;
  const bool valid = warp < tc.TZ && lane < tc.lanes && y < d.ny && z < d.nz;
  const long w = valid ? ((long)z * d.ny + y) * d.wx + wx : 0;
  const uint32_t* Xq = X + q * xs;
  const int32_t* xb = xbox + q * bs;
  const int bx0 = ld_box<kCoh>(xb + 0), by0 = ld_box<kCoh>(xb + 1), bz0 = ld_box<kCoh>(xb + 2);
  const int bx1 = -ld_box<kCoh>(xb + 3), by1 = -ld_box<kCoh>(xb + 4), bz1 = -ld_box<kCoh>(xb + 5);
  const int nwarps = blockDim.x >> 5;
  uint32_t m = 0;
  if (valid) m = (mask ? __ldg(mask + q * ms + w) : 0xffffffffu) & ~__ldg(occ + w);
  // the lane's row of stored edge masks (one word per offset, mstr apart):
  // one address per offset instead of the box index each time
  const uint32_t* mrow = (!kOcc && seg.mask && valid) ? seg.mask + seg.mbox.index(wx, y, z) : nullptr;
  const long mstr = seg.mbox.words();
  const bool touches = bx0 <= bx1 && by1 >= y0 - R && by0 <= y0 + tc.TY - 1 + R &&
                       bz1 >= z0 - R && bz0 <= z0 + tc.TZ - 1 + R;
  if (kOcc)
    for (int i = threadIdx.x; i < tc.TZ + 2 * R; i += blockDim.x) {
      s_ymin[i] = 0x7fffffff;
      s_ymax[i] = -0x7fffffff;
    }
  if (!__syncthreads_or(touches && m != 0)) {
    if (valid) out[q * os + w] = 0u;
    return;
  }
  // Stage the source halo.  The walk below only reads slices inside the z
  // range of the box of X, and rows at most TY - 1 outside its y range (the
  // warp's union of rows), so only that part of the halo is written: words
  // inside the box are copied, the rest of it is zeroed.  A warp writes
  // 32 / P rows per pass, one word per lane.
  {
    const int sz0 = max(bz0, z0 - R), sz1 = min(bz1, z0 + tc.TZ - 1 + R);
    const int sy0 = max(by0 - tc.TY + 1, y0 - R), sy1 = min(by1 + tc.TY - 1, y0 + tc.TY - 1 + R);
    const int ny_rows = sy1 - sy0 + 1, n_rows = (sz1 - sz0 + 1) * ny_rows;
    const int per_pass = 32 / P;
    const int sub = lane / P, c = lane % P, sw = c - 1;
    const bool col_in = sw >= bx0 && sw <= bx1;
    if (ny_rows > 0 && sub < per_pass) {
      for (int r = warp * per_pass + sub; r < n_rows; r += nwarps * per_pass) {
        const int sy = sy0 + r % ny_rows, sz = sz0 + r / ny_rows;
        uint32_t v = 0u;
        if (col_in && sy >= by0 && sy <= by1) v = __ldg(Xq + ((long)sz * d.ny + sy) * d.wx + sw);
        sx[((sz - z0 + R) * RY + (sy - y0 + R)) * P + c] = v;
        if (kOcc) {
          // one lane per staged row records a non-zero row in its slice
          const unsigned nzb = __ballot_sync(__activemask(), v != 0);
          if (c == 0 && ((nzb >> (sub * P)) & ((1u << P) - 1u))) {
            atomicMin(&s_ymin[sz - z0 + R], sy);
            atomicMax(&s_ymax[sz - z0 + R], sy);
          }
        }
      }
    }
  }
  // Without stored edge masks the occupancy halo goes to a second region of
  // the same layout.  A supercover voxel lies between the output voxel and
  // its source, whose z and y lie in the box of X, so only rows between the
  // tile and that box are staged (zero outside the grid).
  uint32_t* so = sx + (tc.TZ + 2 * R) * RY * P;
  if (kOcc) {
    const int oz0 = max(z0 - R, min(z0, bz0)), oz1 = min(z0 + tc.TZ - 1 + R, max(z0 + tc.TZ - 1, bz1));
    const int oy0 = max(y0 - R, min(y0, by0)), oy1 = min(y0 + tc.TY - 1 + R, max(y0 + tc.TY - 1, by1));
    const int ny_rows = oy1 - oy0 + 1, n_rows = (oz1 - oz0 + 1) * ny_rows;
    const int per_pass = 32 / P;
    const int sub = lane / P, c = lane % P, sw = c - 1;
    if (ny_rows > 0 && sub < per_pass) {
      for (int r = warp * per_pass + sub; r < n_rows; r += nwarps * per_pass) {
        const int sy = oy0 + r % ny_rows, sz = oz0 + r / ny_rows;
        uint32_t v = 0u;
        if (sw >= 0 && sw < d.wx && sy >= 0 && sy < d.ny && sz >= 0 && sz < d.nz)
          v = __ldg(seg.occ + ((long)sz * d.ny + sy) * d.wx + sw);
        so[((sz - z0 + R) * RY + (sy - y0 + R)) * P + c] = v;
      }
    }
  }
  __syncthreads();
  uint32_t acc = 0;
  unsigned long long visited = 0, nonzero = 0, mloads = 0, warp_iters = 0;
  if (kCount) {
    // warps that walk the offsets, and their lanes with a non-empty mask
    const unsigned live_lanes = __ballot_sync(kFull, m != 0);
    if (lane == 0 && live_lanes) {
      atomicAdd(counters + 6, 1ull);
      atomicAdd(counters + 7, (unsigned long long)__popc(live_lanes));
    }
  }
  if (__any_sync(kFull, m != 0)) {
    const int side = 2 * R + 1;
    const int ylast = min(y0 + tc.TY, d.ny) - 1;
    const int ez0 = max(bz0 - z, -R), ez1 = min(bz1 - z, R);
    const int ey0 = max(by0 - ylast, -R), ey1 = min(by1 - y0, R);
    // lanes without a word read a harmless in-range spot
    const int base = valid ? ((z - z0 + R) * RY + (y - y0 + R)) * P + (wx + 1) : (R * RY + R) * P + 1;
    bool live = m != 0;
    for (int ez = ez0; ez <= ez1 && ey0 <= ey1; ++ez) {
      // without stored masks (each edge test a supercover walk), only the
      // rows of the source slice that hold a non-zero word
      int eya = ey0, eyb = ey1;
      if (kOcc) {
        const int sl = z - z0 + R + ez;
        eya = max(ey0, s_ymin[sl] - ylast);
        eyb = min(ey1, s_ymax[sl] - y0);
        if (eya > eyb) continue;
      }
      const int32_t* rowp = seg.rows + (ez + R) * side + R;
      const int e1 = __ldg(rowp + eyb + 1);
      const int zb = base + ez * RY * P;
      if (kCount && lane == 0) warp_iters += (unsigned long long)max(0, e1 - __ldg(rowp + eya));
      int e = __ldg(rowp + eya);
      // Eight offsets per pass.  The edge-mask words a pass needs are decided
      // against the accumulator as it stood when the pass began and then
      // loaded together, so their (HBM) latencies overlap instead of each
      // load waiting for the previous one to update the accumulator.
      for (; e + 8 <= e1; e += 8) {
        uint32_t xv[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int32_t t = __ldg(seg.tab + e + i);
          const int a = zb + (t >> 5);
          xv[i] = __funnelshift_r(sx[a], sx[a + 1], t);  // shift taken mod 32
        }
        const uint32_t want = m & ~acc;
        uint32_t any = 0;
#pragma unroll
        for (int i = 0; i < 8; ++i) any |= xv[i];
        if (kCount && live) {
          visited += 8;
#pragma unroll
          for (int i = 0; i < 8; ++i) nonzero += xv[i] != 0;
        }
        if (any & want) {
          if (kOcc) {
            // supercover walks in shared memory: one at a time, each skipped
            // once the accumulator already holds the bits it could add
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              if (xv[i] & m & ~acc) {
                if (kCount) ++mloads;
                acc |= xv[i] & edge_word_tile(seg, e + i, so, base);
              }
            }
          } else {
            uint32_t mv[8];
#pragma unroll
            for (int i = 0; i < 8; ++i)
              mv[i] = (xv[i] & want) ? (mrow ? __ldg(mrow + (long)(e + i) * mstr) : edge_word(d, seg, e + i, w, wx, y, z))
                                     : 0u;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              if (kCount) mloads += (xv[i] & want) != 0;
              acc |= xv[i] & mv[i];
            }
          }
        }
      }
      for (; e < e1; ++e) {
        const int32_t t = __ldg(seg.tab + e);
        const int a = zb + (t >> 5);
        const uint32_t x = __funnelshift_r(sx[a], sx[a + 1], t);
        if (kCount && live) {
          ++visited;
          nonzero += x != 0;
        }
        if (x & m & ~acc) {
          if (kCount) ++mloads;
          acc |= x & (kOcc ? edge_word_tile(seg, e, so, base)
                           : (mrow ? __ldg(mrow + (long)e * mstr) : edge_word(d, seg, e, w, wx, y, z)));
        }
      }
      live = live && (acc & m) != m;
      if (!__any_sync(kFull, live)) break;
    }
  }
  acc &= m;
  if (valid) out[q * os + w] = acc;
  box_accumulate(obox + q * bs, acc != 0, wx, y, z);
  if (kCount && valid) {
    atomicAdd(counters + 0, visited);
    atomicAdd(counters + 1, nonzero);
    atomicAdd(counters + 2, mloads);
    atomicAdd(counters + 3, (unsigned long long)(m != 0));
  }
  if (kCount && lane == 0) atomicAdd(counters + 4, warp_iters);
  if (kCount && threadIdx.x == 0) atomicAdd(counters + 5, 1ull);
}

// The two forms as kernels: with stored edge masks the kernel keeps to 64
// registers (four blocks per SM where shared memory allows); without them
// the supercover walks run better with more registers (three blocks).
template <bool kCount>
__global__ void __launch_bounds__(256) k_propagate_tile(Dims d, SegDev seg, TileCfg tc,
                                                        const uint32_t* __restrict__ X, long xs,
                                                        const uint32_t* __restrict__ mask, long ms,
                                                        const uint32_t* __restrict__ occ,
                                                        uint32_t* __restrict__ out, long os,
                                                        const int32_t* __restrict__ xbox,
                                                        int32_t* __restrict__ obox, long bs,
                                                        unsigned long long* __restrict__ counters) {
  propagate_tile_body<kCount, false>(d, seg, tc, X, xs, mask, ms, occ, out, os, xbox, obox, bs, counters,
                                     blockIdx.y, blockIdx.x);
}

template <bool kCount>
__global__ void __launch_bounds__(256, 3) k_propagate_tile_occ(Dims d, SegDev seg, TileCfg tc,
                                                               const uint32_t* __restrict__ X, long xs,
                                                               const uint32_t* __restrict__ mask, long ms,
                                                               const uint32_t* __restrict__ occ,
                                                               uint32_t* __restrict__ out, long os,
                                                               const int32_t* __restrict__ xbox,
                                                               int32_t* __restrict__ obox, long bs,
                                                               unsigned long long* __restrict__ counters) {
  propagate_tile_body<kCount, true>(d, seg, tc, X, xs, mask, ms, occ, out, os, xbox, obox, bs, counters,
                                    blockIdx.y, blockIdx.x);
}

// The same kernels over a work list of (query, tile) pairs that can hold
// output (built by k_tile_list): a grid of resident blocks walks the list,
// instead of one block per tile of every query -- most of which would find
// nothing to do after staging their masks.
template <bool kCount, bool kOccT>
__device__ __forceinline__ void propagate_list(const Dims& d, const SegDev& seg, const TileCfg& tc,
                                               const uint32_t* X, long xs, const uint32_t* mask, long ms,
                                               const uint32_t* occ, uint32_t* out, long os,
                                               const int32_t* xbox, int32_t* obox, long bs,
                                               unsigned long long* counters, const int2* items,
                                               int* count) {
  // count[0]: items in the list; count[1]: the next item to take (items
  // differ a lot in cost, so blocks take them one at a time)
  __shared__ int s_it;
  const int n = count[0];
  for (;;) {
    __syncthreads();  // the previous item's readers are done with shared memory
    if (threadIdx.x == 0) s_it = atomicAdd(count + 1, 1);
    __syncthreads();
    const int it = s_it;
    if (it >= n) break;
    const int2 t = items[it];
    propagate_tile_body<kCount, kOccT>(d, seg, tc, X, xs, mask, ms, occ, out, os, xbox, obox, bs, counters,
                                       t.x, t.y);
  }
}

template <bool kCount>
__global__ void __launch_bounds__(256) k_propagate_tile_list(Dims d, SegDev seg, TileCfg tc,
                                                             const uint32_t* __restrict__ X, long xs,
                                                             const uint32_t* __restrict__ mask, long ms,
                                                             const uint32_t* __restrict__ occ,
                                                             uint32_t* __restrict__ out, long os,
                                                             const int32_t* __restrict__ xbox,
                                                             int32_t* __restrict__ obox, long bs,
                                                             unsigned long long* __restrict__ counters,
                                                             const int2* __restrict__ items,
                                                             int* __restrict__ count) {
  propagate_list<kCount, false>(d, seg, tc, X, xs, mask, ms, occ, out, os, xbox, obox, bs, counters, items,
                                count);
}

template <bool kCount>
__global__ void __launch_bounds__(256, 3) k_propagate_tile_occ_list(Dims d, SegDev seg, TileCfg tc,
                                                                    const uint32_t* __restrict__ X, long xs,
                                                                    const uint32_t* __restrict__ mask,
                                                                    long ms, const uint32_t* __restrict__ occ,
                                                                    uint32_t* __restrict__ out, long os,
                                                                    const int32_t* __restrict__ xbox,
                                                                    int32_t* __restrict__ obox, long bs,
                                                                    unsigned long long* __restrict__ counters,
                                                                    const int2* __restrict__ items,
                                                                    int* __restrict__ count) {
  propagate_list<kCount, true>(d, seg, tc, X, xs, mask, ms, occ, out, os, xbox, obox, bs, counters, items,
                               count);
}

// Two queries per block.  The queries of a batched backward pass share the
// output mask (F_{k-1} & ~Occ) and every edge-mask word M_e[p]: a block that
// carries queries q0 = 2 blockIdx.y and q1 = q0 + 1 over one tile stages both
// source halos interleaved (one 64-bit shared word per position), decodes
// each offset once, fetches both queries' source words with one 64-bit load
// per word, and loads an edge-mask word once when either query can still
// take bits from it.  The walk covers the union of the two queries' ranges
// (a query's staged words outside its own box are zero).  Stored edge masks
// only; results equal two one-query blocks.
// kCoh: the boxes were written earlier in the same kernel (the persistent
// batch), read with coherent loads.
template <bool kCount, bool kWrap, bool kOcc, bool kCoh>
__device__ __forceinline__ void propagate_pair_body(const Dims& d, const SegDev& seg, const TileCfg& tc,
                                                    const uint32_t* __restrict__ X, long xs,
                                                    const uint32_t* __restrict__ mask,
                                                    const uint32_t* __restrict__ occ,
                                                    uint32_t* __restrict__ out, long os, int Q,
                                                    const int32_t* __restrict__ xbox,
                                                    int32_t* __restrict__ obox, long bs,
                                                    unsigned long long* __restrict__ counters, int tile,
                                                    int pair) {
  extern __shared__ uint2 s2_raw[];
  // kWrap: rows staged at pitch wx without pad words (conflict-free 64-bit
  // loads: a half warp reads 16 consecutive words), one spare word at both
  // ends of the array; the words a row-end lane reads across the row's end
  // belong to the neighbouring row and are masked off below
  uint2* s2 = kWrap ? s2_raw + 1 : s2_raw;
  constexpr unsigned kFull = 0xffffffffu;
  const int q0 = 2 * pair, q1 = q0 + 1;
  const bool has1 = q1 < Q;
  const int y0 = (tile % tc.tiles_y) * tc.TY, z0 = (tile / tc.tiles_y) * tc.TZ;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int R = seg.R, RY = tc.TY + 2 * R, P = kWrap ? d.wx : tc.P;
  const int z = z0 + warp, wx = lane % d.wx, y = y0 + lane / d.wx;
  const bool valid = warp < tc.TZ && lane < tc.lanes && y < d.ny && z < d.nz;
  const long w = valid ? ((long)z * d.ny + y) * d.wx + wx : 0;
  // the boxes of both sources (an empty box for a missing second query)
  int b0[6], b1[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    b0[i] = ld_box<kCoh>(xbox + q0 * bs + i);
    b1[i] = has1 ? ld_box<kCoh>(xbox + q1 * bs + i) : 0x7f7f7f7f;
  }
  const int ax0 = b0[0], ay0 = b0[1], az0 = b0[2], ax1 = -b0[3], ay1 = -b0[4], az1 = -b0[5];
  const int cx0 = b1[0], cy0 = b1[1], cz0 = b1[2], cx1 = -b1[3], cy1 = -b1[4], cz1 = -b1[5];
  auto touches = [&](int x0_, int y0_, int z0_, int x1_, int y1_, int z1_) {
    return x0_ <= x1_ && y1_ >= y0 - R && y0_ <= y0 + tc.TY - 1 + R && z1_ >= z0 - R && z0_ <= z0 + tc.TZ - 1 + R;
  };
  const bool t0 = touches(ax0, ay0, az0, ax1, ay1, az1), t1 = touches(cx0, cy0, cz0, cx1, cy1, cz1);
  uint32_t m = 0;
  if (valid) m = (mask ? __ldg(mask + w) : 0xffffffffu) & ~__ldg(occ + w);
  const uint32_t* mrow = (!kOcc && valid) ? seg.mask + seg.mbox.index(wx, y, z) : nullptr;
  const long mstr = seg.mbox.words();
  if (!__syncthreads_or((t0 || t1) && m != 0)) {
    if (valid) {
      out[q0 * os + w] = 0u;
      if (has1) out[q1 * os + w] = 0u;
    }
    return;
  }
  // the union of the two boxes (an empty box contributes nothing)
  const bool e0 = ax0 > ax1, e1b = cx0 > cx1;
  const int uy0 = e0 ? cy0 : (e1b ? ay0 : min(ay0, cy0)), uy1 = e0 ? cy1 : (e1b ? ay1 : max(ay1, cy1));
  const int uz0 = e0 ? cz0 : (e1b ? az0 : min(az0, cz0)), uz1 = e0 ? cz1 : (e1b ? az1 : max(az1, cz1));
  // stage both halos, interleaved: the rows the walk can read (as in the
  // one-query form, over the union of the boxes), box words copied, the rest zero
  {
    const int sz0 = max(uz0, z0 - R), sz1 = min(uz1, z0 + tc.TZ - 1 + R);
    const int sy0 = max(uy0 - tc.TY + 1, y0 - R), sy1 = min(uy1 + tc.TY - 1, y0 + tc.TY - 1 + R);
    const int ny_rows = sy1 - sy0 + 1, n_rows = (sz1 - sz0 + 1) * ny_rows;
    const int per_pass = 32 / P, nwarps = blockDim.x >> 5;
    const int sub = lane / P, c = lane % P, sw = kWrap ? c : c - 1;
    if (ny_rows > 0 && sub < per_pass) {
      for (int r = warp * per_pass + sub; r < n_rows; r += nwarps * per_pass) {
        const int sy = sy0 + r % ny_rows, sz = sz0 + r / ny_rows;
        const long row = ((long)sz * d.ny + sy) * d.wx + sw;
        uint2 v = make_uint2(0u, 0u);
        if (sw >= ax0 && sw <= ax1 && sy >= ay0 && sy <= ay1 && sz >= az0 && sz <= az1)
          v.x = __ldg(X + q0 * xs + row);
        if (sw >= cx0 && sw <= cx1 && sy >= cy0 && sy <= cy1 && sz >= cz0 && sz <= cz1)
          v.y = __ldg(X + q1 * xs + row);
        s2[((sz - z0 + R) * RY + (sy - y0 + R)) * P + c] = v;
      }
    }
  }
  // kOcc (no stored edge masks): the occupancy halo after the pair halo,
  // same rows and pitch, one word per position; each edge test walks the
  // offset's supercover there, once for both queries.  A supercover voxel
  // lies between the output voxel and its source, so only the rows between
  // the tile and the union box are staged (zero outside the grid).
  uint32_t* so = reinterpret_cast<uint32_t*>(s2 + (tc.TZ + 2 * R) * RY * P);
  if (kOcc) {
    const int oz0 = max(z0 - R, min(z0, uz0)), oz1 = min(z0 + tc.TZ - 1 + R, max(z0 + tc.TZ - 1, uz1));
    const int oy0 = max(y0 - R, min(y0, uy0)), oy1 = min(y0 + tc.TY - 1 + R, max(y0 + tc.TY - 1, uy1));
    const int ny_rows = oy1 - oy0 + 1, n_rows = (oz1 - oz0 + 1) * ny_rows;
    const int per_pass = 32 / P, nwarps = blockDim.x >> 5;
    const int sub = lane / P, c = lane % P, sw = c - 1;
    if (ny_rows > 0 && sub < per_pass) {
      for (int r = warp * per_pass + sub; r < n_rows; r += nwarps * per_pass) {
        const int sy = oy0 + r % ny_rows, sz = oz0 + r / ny_rows;
        uint32_t v = 0u;
        if (sw >= 0 && sw < d.wx && sy >= 0 && sy < d.ny && sz >= 0 && sz < d.nz)
          v = __ldg(seg.occ + ((long)sz * d.ny + sy) * d.wx + sw);
        so[((sz - z0 + R) * RY + (sy - y0 + R)) * P + c] = v;
      }
    }
  }
  __syncthreads();
  uint32_t acc0 = 0, acc1 = 0;
  unsigned long long visited = 0, nonzero = 0, mloads = 0, warp_iters = 0;
  if (__any_sync(kFull, m != 0)) {
    const int side = 2 * R + 1;
    const int ylast = min(y0 + tc.TY, d.ny) - 1;
    const int ez0 = max(uz0 - z, -R), ez1 = min(uz1 - z, R);
    const int ey0 = max(uy0 - ylast, -R), ey1 = min(uy1 - y0, R);
    const int base = valid ? ((z - z0 + R) * RY + (y - y0 + R)) * P + (wx + (kWrap ? 0 : 1))
                           : (R * RY + R) * P + 1;
    // kWrap: the bits a row-end lane would take from across the row's end
    const bool first = wx == 0, last = wx == d.wx - 1;
    auto row_mask = [&](int32_t t) -> uint32_t {
      if (!kWrap) return 0xffffffffu;
      const int sh = t & 31;
      if ((t >> 5) & 1) return first ? 0xffffffffu << (32 - sh) : 0xffffffffu;  // dx = sh - 32 < 0
      return (last && sh) ? 0xffffffffu >> sh : 0xffffffffu;
    };
    bool live0 = m != 0, live1 = has1 && m != 0;
    for (int ez = ez0; ez <= ez1 && ey0 <= ey1; ++ez) {
      const int32_t* rowp = seg.rows + (ez + R) * side + R;
      const int e1 = __ldg(rowp + ey1 + 1);
      const int zb = base + ez * RY * P;
      if (kCount && lane == 0) warp_iters += (unsigned long long)max(0, e1 - __ldg(rowp + ey0));
      int e = __ldg(rowp + ey0);
      for (; e + 8 <= e1; e += 8) {
        uint32_t xa[8], xb[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int32_t t = __ldg((kWrap ? seg.tabw : seg.tab) + e + i);
          const int a = zb + (t >> (kWrap ? 6 : 5));
          const uint2 lo = s2[a], hi = s2[a + 1];
          const uint32_t mk = row_mask(t);
          xa[i] = __funnelshift_r(lo.x, hi.x, t) & mk;  // shift taken mod 32
          xb[i] = __funnelshift_r(lo.y, hi.y, t) & mk;
        }
        const uint32_t want0 = m & ~acc0, want1 = m & ~acc1;
        uint32_t any = 0;
#pragma unroll
        for (int i = 0; i < 8; ++i) any |= (xa[i] & want0) | (xb[i] & want1);
        if (kCount) {
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            if (live0) nonzero += xa[i] != 0;
            if (live1) nonzero += xb[i] != 0;
          }
          visited += 8 * ((int)live0 + (int)live1);
        }
        if (any && kOcc) {
          // supercover walks one at a time, each skipped once both
          // accumulators hold the bits it could add
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            if ((xa[i] & m & ~acc0) | (xb[i] & m & ~acc1)) {
              if (kCount) ++mloads;
              const uint32_t f = edge_word_tile(seg, e + i, so, base);
              acc0 |= xa[i] & f;
              acc1 |= xb[i] & f;
            }
          }
        } else if (any) {
          uint32_t mv[8];
#pragma unroll
          for (int i = 0; i < 8; ++i)
            mv[i] = ((xa[i] & want0) | (xb[i] & want1)) ? __ldg(mrow + (long)(e + i) * mstr) : 0u;
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            if (kCount) mloads += ((xa[i] & want0) | (xb[i] & want1)) != 0;
            acc0 |= xa[i] & mv[i];
            acc1 |= xb[i] & mv[i];
          }
        }
      }
      for (; e < e1; ++e) {
        const int32_t t = __ldg((kWrap ? seg.tabw : seg.tab) + e);
        const int a = zb + (t >> (kWrap ? 6 : 5));
        const uint2 lo = s2[a], hi = s2[a + 1];
        const uint32_t mk = row_mask(t);
        const uint32_t x0 = __funnelshift_r(lo.x, hi.x, t) & mk, x1 = __funnelshift_r(lo.y, hi.y, t) & mk;
        if (kCount) {
          if (live0) {
            ++visited;
            nonzero += x0 != 0;
          }
          if (live1) {
            ++visited;
            nonzero += x1 != 0;
          }
        }
        const uint32_t need = (x0 & m & ~acc0) | (x1 & m & ~acc1);
        if (need) {
          if (kCount) ++mloads;
          const uint32_t mv = kOcc ? edge_word_tile(seg, e, so, base) : __ldg(mrow + (long)e * mstr);
          acc0 |= x0 & mv;
          acc1 |= x1 & mv;
        }
      }
      live0 = live0 && (acc0 & m) != m;
      live1 = live1 && (acc1 & m) != m;
      if (!__any_sync(kFull, live0 || live1)) break;
    }
  }
  acc0 &= m;
  acc1 &= m;
  if (valid) {
    out[q0 * os + w] = acc0;
    if (has1) out[q1 * os + w] = acc1;
  }
  box_accumulate(obox + q0 * bs, acc0 != 0, wx, y, z);
  if (has1) box_accumulate(obox + q1 * bs, acc1 != 0, wx, y, z);
  if (kCount) {
    if (valid) {
      atomicAdd(counters + 0, visited);
      atomicAdd(counters + 1, nonzero);
      atomicAdd(counters + 2, mloads);
      atomicAdd(counters + 3, (unsigned long long)(m != 0) * (has1 ? 2ull : 1ull));
    }
    if (lane == 0) atomicAdd(counters + 4, warp_iters);
    if (threadIdx.x == 0) atomicAdd(counters + 5, 1ull);
  }
}

template <bool kCount, bool kWrap, bool kOcc = false>
__global__ void __launch_bounds__(256) k_propagate_tile_pair(Dims d, SegDev seg, TileCfg tc,
                                                             const uint32_t* __restrict__ X, long xs,
                                                             const uint32_t* __restrict__ mask,
                                                             const uint32_t* __restrict__ occ,
                                                             uint32_t* __restrict__ out, long os, int Q,
                                                             const int32_t* __restrict__ xbox,
                                                             int32_t* __restrict__ obox, long bs,
                                                             unsigned long long* __restrict__ counters) {
  propagate_pair_body<kCount, kWrap, kOcc, false>(d, seg, tc, X, xs, mask, occ, out, os, Q, xbox, obox, bs,
                                                  counters, blockIdx.x, blockIdx.y);
}

// The work list of one propagation: for every query q, the tiles whose
// output words can take bits -- those within reach R (in y and z) of the
// word box of X[q], and inside the box of the output mask when one is given
// (one box for all queries).  One block; items {q, tile} in query order.
__global__ void k_tile_list(Dims d, TileCfg tc, int R, int Q, const int32_t* __restrict__ xbox, long bs,
                            const int32_t* __restrict__ mbox, int2* __restrict__ items, long cap,
                            int* __restrict__ count) {
  __shared__ int warp_sum[32];
  __shared__ long base;
  if (threadIdx.x == 0) base = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  for (int q0 = 0; q0 < Q; q0 += blockDim.x) {
    const int q = q0 + threadIdx.x;
    int ty0 = 0, ty1 = -1, tz0 = 0, tz1 = -1;
    if (q < Q) {
      const int32_t* b = xbox + q * bs;
      const int bx0 = b[0], by0 = b[1], bz0 = b[2], bx1 = -b[3], by1 = -b[4], bz1 = -b[5];
      if (bx0 <= bx1) {
        int ylo = max(0, by0 - R), yhi = min(d.ny - 1, by1 + R);
        int zlo = max(0, bz0 - R), zhi = min(d.nz - 1, bz1 + R);
        if (mbox) {
          if (mbox[0] > -mbox[3]) {
            yhi = -1;  // empty output mask
          } else {
            ylo = max(ylo, mbox[1]);
            yhi = min(yhi, -mbox[4]);
            zlo = max(zlo, mbox[2]);
            zhi = min(zhi, -mbox[5]);
          }
        }
        if (ylo <= yhi && zlo <= zhi) {
          ty0 = ylo / tc.TY;
          ty1 = yhi / tc.TY;
          tz0 = zlo / tc.TZ;
          tz1 = zhi / tc.TZ;
        }
      }
    }
    const int c = max(0, ty1 - ty0 + 1) * max(0, tz1 - tz0 + 1);
    // exclusive prefix sum of c over the block
    int incl = c;
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    if (lane == 31) warp_sum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      int v = lane < nwarp ? warp_sum[lane] : 0;
      for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
      }
      if (lane < nwarp) warp_sum[lane] = v;  // inclusive sums of the warps
    }
    __syncthreads();
    const long off = base + (warp > 0 ? warp_sum[warp - 1] : 0) + (incl - c);
    long k = 0;
    for (int tz = tz0; tz <= tz1; ++tz)
      for (int ty = ty0; ty <= ty1; ++ty, ++k)
        if (off + k < cap) items[off + k] = make_int2(q, tz * tc.tiles_y + ty);
    __syncthreads();
    if (threadIdx.x == 0) base += warp_sum[nwarp - 1];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    count[0] = (int)min(base, cap);
    count[1] = 0;  // the next item to take
  }
}

// The same propagation with a 16-slice tile: warp i computes the output
// words of slices z0 + i and z0 + 8 + i, so each offset's table entry and
// address serve two output words (two shared-memory pairs, two funnel
// shifts).  Slices of the pair outside the z range of the box of X at a
// given dz are masked out (their shared words are not staged).
template <bool kCount>
__global__ void __launch_bounds__(256, 2) k_propagate_tile2(Dims d, SegDev seg, TileCfg tc,
                                                         const uint32_t* __restrict__ X, long xs,
                                                         const uint32_t* __restrict__ mask, long ms,
                                                         const uint32_t* __restrict__ occ,
                                                         uint32_t* __restrict__ out, long os,
                                                         const int32_t* __restrict__ xbox,
                                                         int32_t* __restrict__ obox, long bs,
                                                         unsigned long long* __restrict__ counters) {
  extern __shared__ uint32_t sx[];
  constexpr unsigned kFull = 0xffffffffu;
  constexpr int TD = 16;
  const int q = blockIdx.y;
  const int y0 = (blockIdx.x % tc.tiles_y) * tc.TY, z0 = (blockIdx.x / tc.tiles_y) * TD;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int R = seg.R, RY = tc.TY + 2 * R, P = tc.P;
  const int za = z0 + warp, zb = za + 8, wx = lane % d.wx, y = y0 + lane / d.wx;
  const bool lane_ok = lane < tc.lanes && y < d.ny;
  const bool va = lane_ok && za < d.nz, vb = lane_ok && zb < d.nz;
  const long wa = va ? ((long)za * d.ny + y) * d.wx + wx : 0;
  const long wb = vb ? ((long)zb * d.ny + y) * d.wx + wx : 0;
  const uint32_t* Xq = X + q * xs;
  const int32_t* xb = xbox + q * bs;
  const int bx0 = __ldg(xb + 0), by0 = __ldg(xb + 1), bz0 = __ldg(xb + 2);
  const int bx1 = -__ldg(xb + 3), by1 = -__ldg(xb + 4), bz1 = -__ldg(xb + 5);
  uint32_t ma = 0, mb = 0;
  if (va) ma = (mask ? __ldg(mask + q * ms + wa) : 0xffffffffu) & ~__ldg(occ + wa);
  if (vb) mb = (mask ? __ldg(mask + q * ms + wb) : 0xffffffffu) & ~__ldg(occ + wb);
  const bool touches = bx0 <= bx1 && by1 >= y0 - R && by0 <= y0 + tc.TY - 1 + R &&
                       bz1 >= z0 - R && bz0 <= z0 + TD - 1 + R;
  if (!__syncthreads_or(touches && (ma | mb) != 0)) {
    if (va) out[q * os + wa] = 0u;
    if (vb) out[q * os + wb] = 0u;
    return;
  }
  // stage the readable part of the source halo (as in k_propagate_tile)
  {
    const int sz0 = max(bz0, z0 - R), sz1 = min(bz1, z0 + TD - 1 + R);
    const int sy0 = max(by0 - tc.TY + 1, y0 - R), sy1 = min(by1 + tc.TY - 1, y0 + tc.TY - 1 + R);
    const int ny_rows = sy1 - sy0 + 1, n_rows = (sz1 - sz0 + 1) * ny_rows;
    const int per_pass = 32 / P;
    const int sub = lane / P, c = lane % P, sw = c - 1;
    const bool col_in = sw >= bx0 && sw <= bx1;
    if (ny_rows > 0 && sub < per_pass) {
      for (int r = warp * per_pass + sub; r < n_rows; r += 8 * per_pass) {
        const int sy = sy0 + r % ny_rows, sz = sz0 + r / ny_rows;
        uint32_t v = 0u;
        if (col_in && sy >= by0 && sy <= by1) v = __ldg(Xq + ((long)sz * d.ny + sy) * d.wx + sw);
        sx[((sz - z0 + R) * RY + (sy - y0 + R)) * P + c] = v;
      }
    }
  }
  __syncthreads();
  uint32_t acc_a = 0, acc_b = 0;
  unsigned long long visited = 0, nonzero = 0, mloads = 0, warp_iters = 0;
  if (__any_sync(kFull, (ma | mb) != 0)) {
    const int side = 2 * R + 1;
    const int ylast = min(y0 + tc.TY, d.ny) - 1;
    const int ez0 = max(bz0 - zb, -R), ez1 = min(bz1 - za, R);
    const int ey0 = max(by0 - ylast, -R), ey1 = min(by1 - y0, R);
    const int base_a = lane_ok ? ((warp + R) * RY + (y - y0 + R)) * P + (wx + 1) : (R * RY + R) * P + 1;
    const int slice8 = 8 * RY * P;
    bool live_a = ma != 0, live_b = mb != 0;
    for (int ez = ez0; ez <= ez1 && ey0 <= ey1; ++ez) {
      const bool ua = za + ez >= bz0 && za + ez <= bz1;
      const bool ub = zb + ez >= bz0 && zb + ez <= bz1;
      if (!ua && !ub) continue;
      const uint32_t ka = ua ? 0xffffffffu : 0u, kb = ub ? 0xffffffffu : 0u;
      const int32_t* rowp = seg.rows + (ez + R) * side + R;
      const int e1 = __ldg(rowp + ey1 + 1);
      const int za_b = base_a + ez * RY * P, zb_b = za_b + slice8;
      int e = __ldg(rowp + ey0);
      if (kCount && lane == 0) warp_iters += (unsigned long long)max(0, e1 - e);
      for (; e + 8 <= e1; e += 8) {
        uint32_t xa[8], xb_[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int32_t t = __ldg(seg.tab + e + i);
          const int dl = t >> 5;
          xa[i] = __funnelshift_r(sx[za_b + dl], sx[za_b + dl + 1], t) & ka;
          xb_[i] = __funnelshift_r(sx[zb_b + dl], sx[zb_b + dl + 1], t) & kb;
        }
        const uint32_t want_a = ma & ~acc_a, want_b = mb & ~acc_b;
        uint32_t any_a = 0, any_b = 0;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          any_a |= xa[i];
          any_b |= xb_[i];
        }
        if (kCount) {
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            if (live_a && ua) {
              ++visited;
              nonzero += xa[i] != 0;
            }
            if (live_b && ub) {
              ++visited;
              nonzero += xb_[i] != 0;
            }
          }
        }
        if (any_a & want_a) {
          uint32_t mv[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) mv[i] = (xa[i] & want_a) ? edge_word(d, seg, e + i, wa, wx, y, za) : 0u;
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            if (kCount) mloads += (xa[i] & want_a) != 0;
            acc_a |= xa[i] & mv[i];
          }
        }
        if (any_b & want_b) {
          uint32_t mv[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) mv[i] = (xb_[i] & want_b) ? edge_word(d, seg, e + i, wb, wx, y, zb) : 0u;
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            if (kCount) mloads += (xb_[i] & want_b) != 0;
            acc_b |= xb_[i] & mv[i];
          }
        }
      }
      for (; e < e1; ++e) {
        const int32_t t = __ldg(seg.tab + e);
        const int dl = t >> 5;
        const uint32_t x1 = __funnelshift_r(sx[za_b + dl], sx[za_b + dl + 1], t) & ka;
        const uint32_t x2 = __funnelshift_r(sx[zb_b + dl], sx[zb_b + dl + 1], t) & kb;
        if (kCount) {
          if (live_a && ua) {
            ++visited;
            nonzero += x1 != 0;
          }
          if (live_b && ub) {
            ++visited;
            nonzero += x2 != 0;
          }
        }
        if (x1 & ma & ~acc_a) {
          if (kCount) ++mloads;
          acc_a |= x1 & edge_word(d, seg, e, wa, wx, y, za);
        }
        if (x2 & mb & ~acc_b) {
          if (kCount) ++mloads;
          acc_b |= x2 & edge_word(d, seg, e, wb, wx, y, zb);
        }
      }
      live_a = live_a && (acc_a & ma) != ma;
      live_b = live_b && (acc_b & mb) != mb;
      if (!__any_sync(kFull, live_a || live_b)) break;
    }
  }
  acc_a &= ma;
  acc_b &= mb;
  if (va) out[q * os + wa] = acc_a;
  if (vb) out[q * os + wb] = acc_b;
  box_accumulate(obox + q * bs, acc_a != 0, wx, y, za);
  box_accumulate(obox + q * bs, acc_b != 0, wx, y, zb);
  if (kCount) {
    if (va || vb) {
      atomicAdd(counters + 0, visited);
      atomicAdd(counters + 1, nonzero);
      atomicAdd(counters + 2, mloads);
      atomicAdd(counters + 3, (unsigned long long)(ma != 0) + (unsigned long long)(mb != 0));
    }
    if (lane == 0) atomicAdd(counters + 4, warp_iters);
    if (threadIdx.x == 0) atomicAdd(counters + 5, 1ull);
  }
}

// ------------------------------------------------------------ row lanes

// Row-lane form of the stored-mask propagation, for grids whose rows are at
// most four words (nx <= 128).  A lane owns one whole output row (the WX
// words of one (y, z)); a block covers 32 rows x 8 slices of a tile (the
// helpers below also serve the row-lane edge masks, up to 8-word rows).
// The source halo is staged as (8 + 2R) x (32 + 2R) rows of
// exactly WX words: the words left of x = 0 and right of the row's end are
// zero, so they are not stored, and a warp's 32 lanes read 32 consecutive
// rows with one vector load each, free of bank conflicts.  An offset's
// shifted source row then takes that one load and WX funnel shifts (the
// neighbouring word is the same row's, or zero at its ends); its table
// entry and edge-mask vector serve all WX words of the lane, and with
// NQ = 2 both queries of the block (two planar halos, one output mask).
// The offsets of each dz plane are walked as two runs over the dy range --
// dx < 0, then dx >= 0 (table tabr, row starts rowsr) -- so that every
// batch of offsets shifts the same way.  Results equal the other forms.
template <int WX>
__device__ __forceinline__ void row_ldg(const uint32_t* __restrict__ p, uint32_t (&v)[WX]) {
  if constexpr (WX > 4 && WX % 4 == 0) {
#pragma unroll
    for (int c = 0; c < WX / 4; ++c) {
      const uint4 t = __ldg(reinterpret_cast<const uint4*>(p) + c);
      v[4 * c] = t.x, v[4 * c + 1] = t.y, v[4 * c + 2] = t.z, v[4 * c + 3] = t.w;
    }
  } else if constexpr (WX == 4) {
    const uint4 t = __ldg(reinterpret_cast<const uint4*>(p));
    v[0] = t.x, v[1] = t.y, v[2] = t.z, v[3] = t.w;
  } else if constexpr (WX == 2) {
    const uint2 t = __ldg(reinterpret_cast<const uint2*>(p));
    v[0] = t.x, v[1] = t.y;
  } else {
    v[0] = __ldg(p);
  }
}

template <int WX>
__device__ __forceinline__ void row_lds(const uint32_t* p, uint32_t (&v)[WX]) {
  if constexpr (WX > 4 && WX % 4 == 0) {
#pragma unroll
    for (int c = 0; c < WX / 4; ++c) {
      const uint4 t = reinterpret_cast<const uint4*>(p)[c];
      v[4 * c] = t.x, v[4 * c + 1] = t.y, v[4 * c + 2] = t.z, v[4 * c + 3] = t.w;
    }
  } else if constexpr (WX == 4) {
    const uint4 t = *reinterpret_cast<const uint4*>(p);
    v[0] = t.x, v[1] = t.y, v[2] = t.z, v[3] = t.w;
  } else if constexpr (WX == 2) {
    const uint2 t = *reinterpret_cast<const uint2*>(p);
    v[0] = t.x, v[1] = t.y;
  } else {
    v[0] = *p;
  }
}

template <int WX>
__device__ __forceinline__ void row_st(uint32_t* p, const uint32_t (&v)[WX]) {
  if constexpr (WX > 4 && WX % 4 == 0) {
#pragma unroll
    for (int c = 0; c < WX / 4; ++c)
      reinterpret_cast<uint4*>(p)[c] = make_uint4(v[4 * c], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3]);
  } else if constexpr (WX == 4)
    *reinterpret_cast<uint4*>(p) = make_uint4(v[0], v[1], v[2], v[3]);
  else if constexpr (WX == 2)
    *reinterpret_cast<uint2*>(p) = make_uint2(v[0], v[1]);
  else
    *p = v[0];
}

// The source row shifted by dx (dx & 31 = s): output bit b of word i takes
// source voxel 32 i + b + dx.
template <int WX, bool kNeg>
__device__ __forceinline__ void row_shift(const uint32_t (&v)[WX], int s, uint32_t (&x)[WX]) {
#pragma unroll
  for (int i = 0; i < WX; ++i) {
    if (kNeg)  // dx = s - 32: words i - 1 and i
      x[i] = __funnelshift_r(i > 0 ? v[i > 0 ? i - 1 : 0] : 0u, v[i], s);
    else  // dx = s: words i and i + 1
      x[i] = __funnelshift_r(v[i], i + 1 < WX ? v[i + 1 < WX ? i + 1 : i] : 0u, s);
  }
}

constexpr int kRowTY = 32, kRowTZ = 8, kRowUnits = kRowTY * kRowTZ;
// dynamic shared memory a row-lane block may use (its static arrays take
// up to 3 KiB of the 227 KiB a block may opt in to)
constexpr int kRowSmemMax = 224 * 1024;

// The largest |dy| of an offset in plane dz of a shell with |d|^2 <= hi2
// (at most R).
__device__ __forceinline__ int plane_dy(int dz, int hi2, int R) {
  const int v = max(0, hi2 - dz * dz);
  int r = (int)sqrtf((float)v);
  while ((r + 1) * (r + 1) <= v) ++r;
  while (r * r > v) --r;
  return min(r, R);
}

// Bits r0 .. r0 + len - 1 (r0 < 64, len < 64) of the 96-bit row mask rb[0..2].
__device__ __forceinline__ uint64_t row_window(const uint32_t* rb, int r0, int len) {
  const uint64_t lo = ((uint64_t)rb[1] << 32) | rb[0], hi = rb[2];
  const uint64_t w = r0 == 0 ? lo : ((lo >> r0) | (hi << (64 - r0)));
  return w & ((1ull << len) - 1ull);
}

// The block's output rows are its units: unit t = (slice t / 32, row t %
// 32), each carrying all NQ queries of the block.  Warps take whole planes
// of offsets (dz) from a counter, the larger planes first; for its plane a
// warp lists the units that can still gain bits there (for some query, a
// free voxel not yet reached, and a source row inside the plane's dy reach
// that holds a word, from the per-slice source row masks recorded while
// staging) and walks them 32 per pass, over the dy range of the pass's
// non-empty source rows.  So a saturated row, or one without sources in
// reach, costs no lane.  A unit's accumulators (OR-merged with shared
// atomics: planes may overlap in time, and the OR over planes does not
// depend on their order) and output mask live in shared memory.  The work
// counters' run takes the planes in order with block barriers instead, so
// that its counts do not depend on scheduling.  qfast: blockIdx.x is the
// query pair and blockIdx.y the tile, so the blocks resident together work
// on the same tile and share its edge-mask words in L2.
template <int WX, int NQ, bool kFullBox, bool kCount>
__global__ void __launch_bounds__(256, 2) k_propagate_rows(Dims d, SegDev seg, int tiles_y, int qfast,
                                                           const uint32_t* __restrict__ X, long xs,
                                                           const uint32_t* __restrict__ mask, long ms,
                                                           const uint32_t* __restrict__ occ,
                                                           uint32_t* __restrict__ out, long os, int Q,
                                                           const int32_t* __restrict__ xbox,
                                                           int32_t* __restrict__ obox, long bs,
                                                           unsigned long long* __restrict__ counters) {
  extern __shared__ __align__(16) uint32_t sr[];
  constexpr unsigned kFull = 0xffffffffu;
  constexpr int TY = kRowTY, TZ = kRowTZ, NU = kRowUnits;
  constexpr int kB = NQ == 1 ? 8 : 4;  // offsets per batch
  __shared__ int s_cnt[8], s_next, s_plane[64];
  // per staged slice: the halo rows holding a source word of either query
  __shared__ uint32_t s_rowbits[(kRowTZ + 62) * 3];
  const int tile = qfast ? blockIdx.y : blockIdx.x;
  const int qa = NQ * (qfast ? blockIdx.x : blockIdx.y);
  const int y0 = (tile % tiles_y) * TY, z0 = (tile / tiles_y) * TZ;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int R = seg.R, RY = TY + 2 * R;
  const int HW = (TZ + 2 * R) * RY * WX;  // words of one query's halo
  uint32_t* acc_s = sr + NQ * HW;                          // [NQ][NU][WX]
  uint32_t* m_s = acc_s + NU * NQ * WX;                    // [NU][WX]
  unsigned short* list = reinterpret_cast<unsigned short*>(m_s + NU * WX);  // [8][NU]: per warp
  // the queries' source boxes (an empty box for a missing query)
  int bx0[NQ], by0[NQ], bz0[NQ], bx1[NQ], by1[NQ], bz1[NQ];
  bool has[NQ], touch = false;
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    has[q] = qa + q < Q;
    const int32_t* b = xbox + (long)(qa + q) * bs;
    bx0[q] = has[q] ? __ldg(b + 0) : 0x7f7f7f7f;
    by0[q] = has[q] ? __ldg(b + 1) : 0x7f7f7f7f;
    bz0[q] = has[q] ? __ldg(b + 2) : 0x7f7f7f7f;
    bx1[q] = has[q] ? -__ldg(b + 3) : -0x7f7f7f7f;
    by1[q] = has[q] ? -__ldg(b + 4) : -0x7f7f7f7f;
    bz1[q] = has[q] ? -__ldg(b + 5) : -0x7f7f7f7f;
    touch = touch || (bx0[q] <= bx1[q] && by1[q] >= y0 - R && by0[q] <= y0 + TY - 1 + R &&
                      bz1[q] >= z0 - R && bz0[q] <= z0 + TZ - 1 + R);
  }
  // this thread's row (slice warp, row lane): the output mask, shared by the queries
  const int zt = z0 + warp, yt = y0 + lane;
  const bool valid = yt < d.ny && zt < d.nz;
  const long w0 = valid ? ((long)zt * d.ny + yt) * WX : 0;
  bool m_any = false;
  {
    uint32_t m[WX];
#pragma unroll
    for (int i = 0; i < WX; ++i) m[i] = 0u;
    if (valid) {
      uint32_t o[WX];
      row_ldg<WX>(occ + w0, o);
      if (mask) row_ldg<WX>(mask + (long)qa * ms + w0, m);
#pragma unroll
      for (int i = 0; i < WX; ++i) {
        m[i] = (mask ? m[i] : 0xffffffffu) & ~o[i];
        m_any = m_any || m[i] != 0u;
      }
    }
    row_st<WX>(m_s + threadIdx.x * WX, m);
  }
  for (int i = threadIdx.x; i < (TZ + 2 * R) * 3; i += blockDim.x) s_rowbits[i] = 0u;
  if (!__syncthreads_or(touch && m_any)) {
    if (valid) {
      const uint32_t zero[WX] = {};
#pragma unroll
      for (int q = 0; q < NQ; ++q)
        if (has[q]) row_st<WX>(out + (long)(qa + q) * os + w0, zero);
    }
    return;
  }
  // the union of the boxes in y and z (an empty box contributes nothing)
  int uy0 = 0x7fffffff, uy1 = -0x7fffffff, uz0 = 0x7fffffff, uz1 = -0x7fffffff;
#pragma unroll
  for (int q = 0; q < NQ; ++q)
    if (bx0[q] <= bx1[q]) {
      uy0 = min(uy0, by0[q]), uy1 = max(uy1, by1[q]);
      uz0 = min(uz0, bz0[q]), uz1 = max(uz1, bz1[q]);
    }
  // Stage the halos: the rows the walk can read (slices of the union box in
  // reach, rows at most TY - 1 outside its y range), one row per thread
  // and pass; the words of each query's box are copied, the rest zeroed.
  {
    const int sz0 = max(uz0, z0 - R), sz1 = min(uz1, z0 + TZ - 1 + R);
    const int sy0 = max(uy0 - TY + 1, y0 - R), sy1 = min(uy1 + TY - 1, y0 + TY - 1 + R);
    const int nyr = sy1 - sy0 + 1, nr = (sz1 - sz0 + 1) * nyr;
    if (nyr > 0)
      for (int r = threadIdx.x; r < nr; r += blockDim.x) {
        const int sy = sy0 + r % nyr, sz = sz0 + r / nyr;
        const long row = ((long)sz * d.ny + sy) * WX;
        uint32_t* dst = sr + ((sz - z0 + R) * RY + (sy - y0 + R)) * WX;
        uint32_t nz = 0u;
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
          uint32_t v[WX];
#pragma unroll
          for (int i = 0; i < WX; ++i) v[i] = 0u;
          if (sy >= by0[q] && sy <= by1[q] && sz >= bz0[q] && sz <= bz1[q]) {
            row_ldg<WX>(X + (long)(qa + q) * xs + row, v);
#pragma unroll
            for (int i = 0; i < WX; ++i)
              if (i < bx0[q] || i > bx1[q]) v[i] = 0u;
          }
#pragma unroll
          for (int i = 0; i < WX; ++i) nz |= v[i];
          row_st<WX>(dst + q * HW, v);
        }
        if (nz) {
          const int hr = sy - y0 + R;
          atomicOr(s_rowbits + (sz - z0 + R) * 3 + (hr >> 5), 1u << (hr & 31));
        }
      }
    const uint32_t zero[WX] = {};
#pragma unroll
    for (int q = 0; q < NQ; ++q) row_st<WX>(acc_s + (q * NU + threadIdx.x) * WX, zero);
  }
  __syncthreads();
  unsigned long long visited = 0, nonzero = 0, mloads = 0, warp_iters = 0, passes = 0, pass_lanes = 0;
  const int side = 2 * R + 2;  // row starts per (dz, sign) run, with its end
  const int mx0 = kFullBox ? 0 : seg.mbox.wx0;
  const unsigned mstr = (unsigned)seg.mbox.words();
  const int EZ0 = max(uz0 - (z0 + TZ - 1), -R), EZ1 = min(uz1 - z0, R);
  // One pass of a warp: the units lst[p .. p + 31] (of n_act) over plane
  // ez.  merge: other warps may add to the same units meanwhile (their
  // accumulators are OR-merged into shared memory); else the units are this
  // pass's alone.
  auto do_pass = [&](int ez, const unsigned short* lst, int n_act, int p, bool merge) {
    const bool hasu = p + lane < n_act;
    const int t = hasu ? lst[p + lane] : 0;
    const int zu = z0 + t / 32, yu = y0 + t % 32;
    uint32_t acc[NQ][WX], acc0[NQ][WX], m[WX];
    row_lds<WX>(m_s + t * WX, m);
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      row_lds<WX>(acc_s + (q * NU + t) * WX, acc[q]);
#pragma unroll
      for (int i = 0; i < WX; ++i) acc0[q][i] = acc[q][i];
    }
    if (!hasu)
#pragma unroll
      for (int i = 0; i < WX; ++i) m[i] = 0u;
    // the pass's union of the lanes' dy ranges
    // the pass's union of the lanes' dy ranges: the rows of each lane's
    // window (dy in [-R, R]) that hold a source word
    int lo_dy = 0x7fffffff, hi_dy = -0x7fffffff;
    if (hasu) {
      const int dyx = plane_dy(ez, seg.hi2, R);
      const uint64_t win = row_window(s_rowbits + (zu - z0 + R + ez) * 3, yu - y0 + R - dyx, 2 * dyx + 1);
      if (win) {
        lo_dy = __ffsll((long long)win) - 1 - dyx;
        hi_dy = 63 - __clzll((long long)win) - dyx;
      }
    }
    const int ey0 = __reduce_min_sync(kFull, lo_dy);
    const int ey1 = __reduce_max_sync(kFull, hi_dy);
    const uint32_t* hz = sr + ((zu - z0 + R + ez) * RY + (yu - y0 + R)) * WX;
    const uint32_t* mrow = seg.mask + (hasu ? seg.mbox.index(mx0, yu, zu) : 0);
    // words still open at the pass's start (work counters only)
    unsigned lw = 0;
    if (kCount) {
#pragma unroll
      for (int q = 0; q < NQ; ++q)
#pragma unroll
        for (int i = 0; i < WX; ++i) lw |= (unsigned)((acc[q][i] & m[i]) != m[i]) << (q * WX + i);
      if (lane == 0) {
        ++passes;
        pass_lanes += (unsigned long long)min(32, n_act - p);
      }
    }
    // hz32: the lane's row at dy = -32 (the table stores dy + 32)
    const uint32_t* hz32 = hz - 32 * WX;
    // NB offsets from e on, all shifting the same way
    auto batch = [&](auto neg_tag, auto nb_tag, int e) {
      constexpr bool kNeg = decltype(neg_tag)::value;
      constexpr int NB = decltype(nb_tag)::value;
      uint32_t x[NB][NQ][WX];
      int32_t tb[NB];
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        tb[b] = __ldg(seg.tabr + e + b);
        const uint32_t* p2 = hz32 + ((tb[b] >> 5) & 63) * WX;
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
          uint32_t v[WX];
          row_lds<WX>(p2 + q * HW, v);
          row_shift<WX, kNeg>(v, tb[b] & 31, x[b][q]);
        }
      }
      uint32_t want[NQ][WX];
#pragma unroll
      for (int q = 0; q < NQ; ++q)
#pragma unroll
        for (int i = 0; i < WX; ++i) want[q][i] = m[i] & ~acc[q][i];
      // need[b][i]: the bits offset b could add to word i of some query;
      // with masks over whole rows only their union decides the load
      constexpr int NW = kFullBox ? 1 : WX;
      uint32_t need[NB][NW], any = 0u;
#pragma unroll
      for (int b = 0; b < NB; ++b) {
#pragma unroll
        for (int j = 0; j < NW; ++j) need[b][j] = 0u;
#pragma unroll
        for (int q = 0; q < NQ; ++q)
#pragma unroll
          for (int i = 0; i < WX; ++i) need[b][kFullBox ? 0 : i] |= x[b][q][i] & want[q][i];
#pragma unroll
        for (int j = 0; j < NW; ++j) any |= need[b][j];
      }
      if (kCount) {
        visited += (unsigned long long)NB * __popc(lw);
#pragma unroll
        for (int b = 0; b < NB; ++b)
#pragma unroll
          for (int q = 0; q < NQ; ++q)
#pragma unroll
            for (int i = 0; i < WX; ++i) nonzero += ((lw >> (q * WX + i)) & 1u) && x[b][q][i] != 0u;
      }
      if (any) {
        uint32_t mv[NB][WX];
#pragma unroll
        for (int b = 0; b < NB; ++b) {
          const uint32_t* mp = mrow + (size_t)((unsigned)tb[b] >> 11) * mstr;
          if (kFullBox) {
            if (need[b][0]) {
              row_ldg<WX>(mp, mv[b]);
              if (kCount) mloads += WX;
            } else {
#pragma unroll
              for (int i = 0; i < WX; ++i) mv[b][i] = 0u;
            }
          } else {
#pragma unroll
            for (int i = 0; i < WX; ++i) {
              mv[b][i] = need[b][kFullBox ? 0 : i] ? __ldg(mp + (i - mx0)) : 0u;
              if (kCount) mloads += need[b][kFullBox ? 0 : i] != 0u;
            }
          }
        }
#pragma unroll
        for (int b = 0; b < NB; ++b)
#pragma unroll
          for (int q = 0; q < NQ; ++q)
#pragma unroll
            for (int i = 0; i < WX; ++i) acc[q][i] |= x[b][q][i] & mv[b][i];
      }
    };
    auto run = [&](auto neg_tag, int e, int e1) {
      for (; e + kB <= e1; e += kB) batch(neg_tag, std::integral_constant<int, kB>{}, e);
      for (; e < e1; ++e) batch(neg_tag, std::integral_constant<int, 1>{}, e);
    };
    if (ey0 <= ey1) {
      const int32_t* rs = seg.rowsr + (ez + R) * 2 * side + R;
      const int n0 = __ldg(rs + ey0), n1 = __ldg(rs + ey1 + 1);
      const int p0 = __ldg(rs + side + ey0), p1 = __ldg(rs + side + ey1 + 1);
      if (kCount && lane == 0) warp_iters += (unsigned long long)(n1 - n0 + p1 - p0);
      run(std::true_type{}, n0, n1);
      run(std::false_type{}, p0, p1);
    }
    if (hasu) {
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        if (merge) {
#pragma unroll
          for (int i = 0; i < WX; ++i)
            if (acc[q][i] & ~acc0[q][i]) atomicOr(acc_s + (q * NU + t) * WX + i, acc[q][i]);
        } else {
          row_st<WX>(acc_s + (q * NU + t) * WX, acc[q]);
        }
      }
    }
  };
  if (kCount) {
    // the work counters count in plane order: the block takes each plane
    // together (warps split its open units), with barriers between planes
    for (int ez = EZ0; ez <= EZ1; ++ez) {
      bool act = false;
      {
        uint32_t m[WX];
        row_lds<WX>(m_s + threadIdx.x * WX, m);
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
          uint32_t a[WX];
          row_lds<WX>(acc_s + (q * NU + threadIdx.x) * WX, a);
          bool open = false;
#pragma unroll
          for (int i = 0; i < WX; ++i) open = open || (a[i] & m[i]) != m[i];
          act = act || (open && zt + ez >= bz0[q] && zt + ez <= bz1[q]);
        }
      }
      {
        const int dyx = plane_dy(ez, seg.hi2, R);
        act = act && row_window(s_rowbits + (warp + R + ez) * 3, lane + R - dyx, 2 * dyx + 1) != 0ull;
      }
      const unsigned bal = __ballot_sync(kFull, act);
      if (lane == 0) s_cnt[warp] = __popc(bal);
      __syncthreads();
      int n_act = 0, pos = __popc(bal & ((1u << lane) - 1u));
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        n_act += s_cnt[c];
        pos += c < warp ? s_cnt[c] : 0;
      }
      if (act) list[pos] = (unsigned short)threadIdx.x;
      __syncthreads();
      for (int p = warp * 32; p < n_act; p += 256) do_pass(ez, list, n_act, p, false);
      __syncthreads();
    }
  } else {
    // Warps take whole planes from a counter, the larger ones (nearest
    // dz = 0) first, and each lists the units open for its plane: no block
    // barrier between planes.  A unit's accumulator may lag bits that
    // another warp is adding in another plane; it only gates loads, and the
    // OR of all planes is the same in any order.
    const int n_planes = EZ1 - EZ0 + 1;
    if (threadIdx.x == 0) {
      s_next = 0;
      const int c = min(max(0, EZ0), EZ1);
      int n = 0;
      for (int k = 0; n < n_planes; ++k) {
        if (c + k <= EZ1) s_plane[n++] = c + k;
        if (k > 0 && c - k >= EZ0) s_plane[n++] = c - k;
      }
    }
    __syncthreads();
    unsigned short* wl = list + warp * NU;
    for (;;) {
      int i = 0;
      if (lane == 0) i = atomicAdd(&s_next, 1);
      i = __shfl_sync(kFull, i, 0);
      if (i >= n_planes) break;
      const int ez = s_plane[i];
      const int dyx = plane_dy(ez, seg.hi2, R);  // the plane's rows reach |dy| <= dyx
      int n_act = 0;
      for (int c = 0; c < TZ; ++c) {
        const int t = c * 32 + lane;
        bool act = false;
        uint32_t m[WX];
        row_lds<WX>(m_s + t * WX, m);
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
          uint32_t a[WX];
          row_lds<WX>(acc_s + (q * NU + t) * WX, a);
          bool open = false;
#pragma unroll
          for (int k = 0; k < WX; ++k) open = open || (a[k] & m[k]) != m[k];
          act = act || (open && z0 + c + ez >= bz0[q] && z0 + c + ez <= bz1[q]);
        }
        act = act && row_window(s_rowbits + (c + R + ez) * 3, lane + R - dyx, 2 * dyx + 1) != 0ull;
        const unsigned bal = __ballot_sync(kFull, act);
        if (act) wl[n_act + __popc(bal & ((1u << lane) - 1u))] = (unsigned short)t;
        n_act += __popc(bal);
      }
      __syncwarp();
      for (int p = 0; p < n_act; p += 32) do_pass(ez, wl, n_act, p, true);
      __syncwarp();
    }
    __syncthreads();
  }
  // outputs: this thread's row for each query
  uint32_t m[WX];
  row_lds<WX>(m_s + threadIdx.x * WX, m);
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    if (!has[q]) continue;
    uint32_t acc[WX];
    row_lds<WX>(acc_s + (q * NU + threadIdx.x) * WX, acc);
    int lo = WX, hi = -1;
#pragma unroll
    for (int i = 0; i < WX; ++i) {
      acc[i] &= m[i];
      if (acc[i]) lo = min(lo, i), hi = i;
    }
    if (valid) row_st<WX>(out + (long)(qa + q) * os + w0, acc);
    // the output's box: the lane's first and last non-zero word
    int32_t* box = obox + (long)(qa + q) * bs;
    const bool nz = hi >= 0;
    if (__ballot_sync(kFull, nz)) {
      const int big = 0x7fffffff;
      const int v0 = __reduce_min_sync(kFull, nz ? lo : big);
      const int v1 = __reduce_min_sync(kFull, nz ? yt : big);
      const int v3 = __reduce_min_sync(kFull, nz ? -hi : big);
      const int v4 = __reduce_min_sync(kFull, nz ? -yt : big);
      if (lane == 0) {
        atomicMin(box + 0, v0);
        atomicMin(box + 1, v1);
        atomicMin(box + 2, zt);
        atomicMin(box + 3, v3);
        atomicMin(box + 4, v4);
        atomicMin(box + 5, -zt);
      }
    }
  }
  if (kCount) {
    atomicAdd(counters + 0, visited);
    atomicAdd(counters + 1, nonzero);
    atomicAdd(counters + 2, mloads);
    if (valid) {
      unsigned long long live_words = 0;
#pragma unroll
      for (int i = 0; i < WX; ++i) live_words += m[i] != 0u;
      int nq = 0;
#pragma unroll
      for (int q = 0; q < NQ; ++q) nq += has[q];
      atomicAdd(counters + 3, live_words * nq);
    }
    if (lane == 0) {
      atomicAdd(counters + 4, warp_iters);
      atomicAdd(counters + 6, passes);
      atomicAdd(counters + 7, pass_lanes);
    }
    if (threadIdx.x == 0) atomicAdd(counters + 5, 1ull);
  }
}

// Edge masks with row lanes (rows of 1, 2 or 4 words, reach at most 31): a
// lane owns one row of the mask box, a block 32 rows x 8 slices.  The tile's
// occupancy halo is staged at a pitch of exactly WX words (words outside the
// grid are free, and a segment between two voxels of the grid never leaves
// it), and each supercover voxel of an offset costs the lane one vector load
// of shared memory and WX funnel shifts.  The voxels of one supercover are
// the same for every lane, so the sign of their shift is warp-uniform.
// sctabr[i] = ((vz * (32 + 2R) + vy) << 6) | (vx + 32).  Results equal
// k_edge_masks_tile.
template <int WX, bool kFull>
__global__ void __launch_bounds__(256) k_edge_masks_rows(Dims d, MaskBox b, int tiles_y, int R, int n_off,
                                                         const uint32_t* __restrict__ occ,
                                                         const int32_t* __restrict__ sc_start,
                                                         const int32_t* __restrict__ sctabr,
                                                         uint32_t* __restrict__ mask) {
  extern __shared__ __align__(16) uint32_t so[];
  constexpr int TY = kRowTY, TZ = kRowTZ;
  const int y0 = b.y0 + (blockIdx.x % tiles_y) * TY, z0 = b.z0 + (blockIdx.x / tiles_y) * TZ;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int RY = TY + 2 * R, RZ = TZ + 2 * R;
  for (int r = threadIdx.x; r < RZ * RY; r += blockDim.x) {
    const int sy = y0 - R + r % RY, sz = z0 - R + r / RY;
    uint32_t v[WX];
#pragma unroll
    for (int i = 0; i < WX; ++i) v[i] = 0u;
    if (sy >= 0 && sy < d.ny && sz >= 0 && sz < d.nz) row_ldg<WX>(occ + ((long)sz * d.ny + sy) * WX, v);
    row_st<WX>(so + r * WX, v);
  }
  __syncthreads();
  const int y = y0 + lane, z = z0 + warp;
  if (y > b.y1 || z > b.z1) return;
  const uint32_t* base = so + ((warp + R) * RY + (lane + R)) * WX;
  const long nb = b.words();
  uint32_t* mrow = mask + b.index(b.wx0, y, z);
  const int e_end = min(n_off, (int)(blockIdx.y + 1) * kMaskChunk);
  for (int e = blockIdx.y * kMaskChunk; e < e_end; ++e) {
    const int i1 = __ldg(sc_start + e + 1);
    uint32_t blk[WX];
#pragma unroll
    for (int i = 0; i < WX; ++i) blk[i] = 0u;
#pragma unroll 4
    for (int i = __ldg(sc_start + e); i < i1; ++i) {
      const int32_t t = __ldg(sctabr + i);
      uint32_t v[WX], x[WX];
      row_lds<WX>(base + (t >> 6) * WX, v);
      const int vx = (t & 63) - 32;
      if (vx < 0)
        row_shift<WX, true>(v, vx & 31, x);
      else
        row_shift<WX, false>(v, vx, x);
#pragma unroll
      for (int w = 0; w < WX; ++w) blk[w] |= x[w];
    }
    uint32_t* dst = mrow + (long)e * nb;
    if (kFull) {
      uint32_t o[WX];
#pragma unroll
      for (int w = 0; w < WX; ++w) o[w] = ~blk[w];
      row_st<WX>(dst, o);
    } else {
#pragma unroll
      for (int w = 0; w < WX; ++w)
        if (w >= b.wx0 && w <= b.wx1) dst[w - b.wx0] = ~blk[w];
    }
  }
}

template <int WX>
cudaError_t launch_edge_masks_rows_w(const Dims& d, const MaskBox& b, int R, int n, const uint32_t* occ,
                                     const ShellDev& s, uint32_t* mask, cudaStream_t st) {
  const int tiles_y = (b.nyy() + kRowTY - 1) / kRowTY, tiles_z = (b.z1 - b.z0 + kRowTZ) / kRowTZ;
  const dim3 grid(tiles_y * tiles_z, (n + kMaskChunk - 1) / kMaskChunk);
  const size_t smem = (size_t)(kRowTZ + 2 * R) * (kRowTY + 2 * R) * WX * 4;
  const bool full = b.wx0 == 0 && b.wx1 == d.wx - 1 && ((uintptr_t)mask & ((WX < 4 ? WX : 4) * 4 - 1)) == 0;
  if (full)
    k_edge_masks_rows<WX, true><<<grid, 256, smem, st>>>(d, b, tiles_y, R, n, occ, s.d_sc_start, s.d_sctabr, mask);
  else
    k_edge_masks_rows<WX, false><<<grid, 256, smem, st>>>(d, b, tiles_y, R, n, occ, s.d_sc_start, s.d_sctabr,
                                                          mask);
  return cudaGetLastError();
}

// The row-lane edge masks where they apply (*done = false: use another form).
cudaError_t launch_edge_masks_rows(const Dims& d, const TileCfg& tc, const uint32_t* occ, const ShellDev& s,
                                   const MaskBox& b, uint32_t* mask, cudaStream_t st, bool* done) {
  *done = false;
  const int n = (int)s.host.off.size(), R = s.reach;
  if (!tc.rows || !s.d_sctabr || R > 31 || (d.wx != 1 && d.wx != 2 && d.wx != 4 && d.wx != 8)) return cudaSuccess;
  if (((uintptr_t)occ & (std::min(d.wx, 4) * 4 - 1)) != 0) return cudaSuccess;
  if ((size_t)(kRowTZ + 2 * R) * (kRowTY + 2 * R) * d.wx * 4 > (size_t)kTileOccSmemMax) return cudaSuccess;
  *done = true;
  if (d.wx == 8) return launch_edge_masks_rows_w<8>(d, b, R, n, occ, s, mask, st);
  if (d.wx == 4) return launch_edge_masks_rows_w<4>(d, b, R, n, occ, s, mask, st);
  if (d.wx == 2) return launch_edge_masks_rows_w<2>(d, b, R, n, occ, s, mask, st);
  return launch_edge_masks_rows_w<1>(d, b, R, n, occ, s, mask, st);
}

size_t rows_smem_bytes(int wx, int R, int nq) {
  if (R > 31 || (wx != 1 && wx != 2 && wx != 4)) return 0;
  // the halos, the units' accumulators and output masks, the unit list
  const size_t bytes = (size_t)nq * (kRowTZ + 2 * R) * (kRowTY + 2 * R) * wx * 4 +
                       (size_t)(nq + 1) * kRowUnits * wx * 4 + (size_t)8 * kRowUnits * 2;
  return bytes <= (size_t)kRowSmemMax ? bytes : 0;
}

template <int WX, int NQ, bool kFullBox>
cudaError_t launch_rows_t(const Dims& d, const SegDev& seg, const uint32_t* X, long xs, const uint32_t* mask,
                          long ms, const uint32_t* occ, uint32_t* out, long os, int Q, const int32_t* xbox,
                          int32_t* obox, long bs, cudaStream_t st, unsigned long long* counters, size_t smem) {
  const int tiles_y = (d.ny + kRowTY - 1) / kRowTY, tiles_z = (d.nz + kRowTZ - 1) / kRowTZ;
  const int tiles = tiles_y * tiles_z, groups = (Q + NQ - 1) / NQ;
  // the query groups of one tile next to each other where the grid allows
  const int qfast = tiles <= 65535 ? 1 : 0;
  const dim3 grid = qfast ? dim3(groups, tiles) : dim3(tiles, groups);
  if (counters)
    k_propagate_rows<WX, NQ, kFullBox, true><<<grid, 256, smem, st>>>(d, seg, tiles_y, qfast, X, xs, mask, ms, occ,
                                                                     out, os, Q, xbox, obox, bs, counters);
  else
    k_propagate_rows<WX, NQ, kFullBox, false><<<grid, 256, smem, st>>>(d, seg, tiles_y, qfast, X, xs, mask, ms,
                                                                      occ, out, os, Q, xbox, obox, bs, nullptr);
  return cudaGetLastError();
}

template <int WX>
cudaError_t launch_rows_w(int nq, bool full, const Dims& d, const SegDev& seg, const uint32_t* X, long xs,
                          const uint32_t* mask, long ms, const uint32_t* occ, uint32_t* out, long os, int Q,
                          const int32_t* xbox, int32_t* obox, long bs, cudaStream_t st,
                          unsigned long long* counters, size_t smem) {
  if (nq == 2)
    return full ? launch_rows_t<WX, 2, true>(d, seg, X, xs, mask, ms, occ, out, os, Q, xbox, obox, bs, st, counters, smem)
                : launch_rows_t<WX, 2, false>(d, seg, X, xs, mask, ms, occ, out, os, Q, xbox, obox, bs, st, counters, smem);
  return full ? launch_rows_t<WX, 1, true>(d, seg, X, xs, mask, ms, occ, out, os, Q, xbox, obox, bs, st, counters, smem)
              : launch_rows_t<WX, 1, false>(d, seg, X, xs, mask, ms, occ, out, os, Q, xbox, obox, bs, st, counters, smem);
}

template <int WX>
cudaError_t set_rows_attributes() {
  cudaError_t e = cudaSuccess;
  const void* fns[] = {(const void*)k_propagate_rows<WX, 1, false, false>, (const void*)k_propagate_rows<WX, 1, false, true>,
                       (const void*)k_propagate_rows<WX, 1, true, false>,  (const void*)k_propagate_rows<WX, 1, true, true>,
                       (const void*)k_propagate_rows<WX, 2, false, false>, (const void*)k_propagate_rows<WX, 2, false, true>,
                       (const void*)k_propagate_rows<WX, 2, true, false>,  (const void*)k_propagate_rows<WX, 2, true, true>};
  for (const void* f : fns)
    if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, kRowSmemMax);
  return e;
}

// Queries per block of the row-lane form for a launch, 0 where it does not
// apply: stored edge masks, a batch of two or more queries (a single query,
// the forward sets, measured faster on the other forms), rows of 1, 2 or 4
// words, every row of every set aligned to its width, reach at most 31.
int rows_queries(const Dims& d, const TileCfg& tc, const SegDev& seg, const uint32_t* X, long xs,
                 const uint32_t* mask, long ms, const uint32_t* occ, const uint32_t* out, long os, int Q) {
  if (!tc.rows || !seg.mask || !seg.tabr || !seg.rowsr || Q < 2) return 0;
  const int wx = d.wx;
  if (wx != 1 && wx != 2 && wx != 4) return 0;
  const uintptr_t al = (uintptr_t)wx * 4 - 1;
  if (((uintptr_t)X & al) || ((uintptr_t)out & al) || ((uintptr_t)mask & al) || ((uintptr_t)occ & al)) return 0;
  if (xs % wx || os % wx || (mask && ms % wx)) return 0;
  const int nq = (tc.pair && Q >= 2 && ms == 0) ? 2 : 1;
  return rows_smem_bytes(wx, seg.R, nq) > 0 ? nq : 0;
}

size_t tile2_smem_bytes(const TileCfg& tc, int R) {
  if (R > 31 || tc.P > 31) return 0;
  const size_t bytes = (size_t)(16 + 2 * R) * (tc.TY + 2 * R) * tc.P * 4;
  return bytes <= 200 * 1024 ? bytes : 0;
}

bool propagate_listed(const TileCfg& tc, const SegDev& seg, int Q, long out_stride, const WorkList* wl) {
  if (!wl || Q < kListMinQueries || out_stride <= 0 || tc.depth == 16 || !seg.tab) return false;
  if (wl->cap < (long)Q * tc.tiles_y * tc.tiles_z) return false;
  const size_t smem_o = (!seg.mask && seg.sctab) ? tile_occ_smem_bytes(tc, seg.R) : 0;
  return smem_o > 0 || tile_smem_bytes(tc, seg.R) > 0;
}

cudaError_t launch_tile_list(const Dims& d, const TileCfg& tc, int R, int Q, const int32_t* xbox,
                             long box_stride, const int32_t* mbox, uint32_t* out, long out_stride,
                             const WorkList& wl, cudaStream_t st) {
  // the blocks write only the listed tiles: the rest of every output is zero
  cudaError_t e = cudaMemset2DAsync(out, (size_t)out_stride * 4, 0, (size_t)d.nw * 4, (size_t)Q, st);
  if (e != cudaSuccess) return e;
  k_tile_list<<<1, 1024, 0, st>>>(d, tc, R, Q, xbox, box_stride, mbox, wl.items, (long)Q * tc.tiles_y * tc.tiles_z,
                                  wl.count);
  return cudaGetLastError();
}

cudaError_t launch_propagate(const Dims& d, const TileCfg& tc, const SegDev& seg, const uint32_t* X,
                             long x_stride, const uint32_t* mask, long mask_stride,
                             const uint32_t* occ, uint32_t* out, long out_stride, int Q,
                             const int32_t* xbox, int32_t* obox, long box_stride, cudaStream_t st,
                             unsigned long long* counters, const WorkList* wl) {
  if (Q <= 0) return cudaSuccess;
  // the batched form over a work list that launch_tile_list has built
  const bool listed = propagate_listed(tc, seg, Q, out_stride, wl);
  const int list_grid = (int)std::min<long>((long)Q * tc.tiles_y * tc.tiles_z, wl ? wl->blocks : 1);
  const size_t smem2 = tc.depth == 16 ? tile2_smem_bytes(tc, seg.R) : 0;
  if (smem2 > 0 && seg.tab) {
    dim3 grid(tc.tiles_y * ((d.nz + 15) / 16), Q);
    if (counters)
      k_propagate_tile2<true><<<grid, 256, smem2, st>>>(d, seg, tc, X, x_stride, mask, mask_stride, occ,
                                                        out, out_stride, xbox, obox, box_stride, counters);
    else
      k_propagate_tile2<false><<<grid, 256, smem2, st>>>(d, seg, tc, X, x_stride, mask, mask_stride, occ,
                                                         out, out_stride, xbox, obox, box_stride, nullptr);
    return cudaGetLastError();
  }
  const size_t smem_o = (!seg.mask && seg.sctab) ? tile_occ_smem_bytes(tc, seg.R) : 0;
  if (smem_o > 0 && seg.tab && listed) {
    if (counters)
      k_propagate_tile_occ_list<true><<<list_grid, 256, smem_o, st>>>(
          d, seg, tc, X, x_stride, mask, mask_stride, occ, out, out_stride, xbox, obox, box_stride, counters,
          wl->items, wl->count);
    else
      k_propagate_tile_occ_list<false><<<list_grid, 256, smem_o, st>>>(
          d, seg, tc, X, x_stride, mask, mask_stride, occ, out, out_stride, xbox, obox, box_stride, nullptr,
          wl->items, wl->count);
    return cudaGetLastError();
  }
  // two queries per block without stored masks: the pair halo and the
  // occupancy halo, the supercover walks shared by both queries
  if (smem_o > 0 && seg.tab && Q >= 2 && tc.pair && mask_stride == 0 && 3 * (smem_o / 2) <= (size_t)kTileOccSmemMax) {
    dim3 grid(tc.tiles_y * tc.tiles_z, (Q + 1) / 2);
    if (counters)
      k_propagate_tile_pair<true, false, true><<<grid, 256, 3 * (smem_o / 2), st>>>(
          d, seg, tc, X, x_stride, mask, occ, out, out_stride, Q, xbox, obox, box_stride, counters);
    else
      k_propagate_tile_pair<false, false, true><<<grid, 256, 3 * (smem_o / 2), st>>>(
          d, seg, tc, X, x_stride, mask, occ, out, out_stride, Q, xbox, obox, box_stride, nullptr);
    return cudaGetLastError();
  }
  if (smem_o > 0 && seg.tab) {
    dim3 grid(tc.tiles_y * tc.tiles_z, Q);
    if (counters)
      k_propagate_tile_occ<true><<<grid, 256, smem_o, st>>>(d, seg, tc, X, x_stride, mask, mask_stride,
                                                              occ, out, out_stride, xbox, obox, box_stride,
                                                              counters);
    else
      k_propagate_tile_occ<false><<<grid, 256, smem_o, st>>>(d, seg, tc, X, x_stride, mask, mask_stride,
                                                               occ, out, out_stride, xbox, obox, box_stride,
                                                               nullptr);
    return cudaGetLastError();
  }
  if (!listed) {
    const int nq = rows_queries(d, tc, seg, X, x_stride, mask, mask_stride, occ, out, out_stride, Q);
    if (nq) {
      const size_t smem_r = rows_smem_bytes(d.wx, seg.R, nq);
      const bool full = seg.mbox.wx0 == 0 && seg.mbox.wx1 == d.wx - 1;
      if (d.wx == 4)
        return launch_rows_w<4>(nq, full, d, seg, X, x_stride, mask, mask_stride, occ, out, out_stride, Q, xbox,
                                obox, box_stride, st, counters, smem_r);
      if (d.wx == 2)
        return launch_rows_w<2>(nq, full, d, seg, X, x_stride, mask, mask_stride, occ, out, out_stride, Q, xbox,
                                obox, box_stride, st, counters, smem_r);
      return launch_rows_w<1>(nq, full, d, seg, X, x_stride, mask, mask_stride, occ, out, out_stride, Q, xbox,
                              obox, box_stride, st, counters, smem_r);
    }
  }
  const size_t smem = tile_smem_bytes(tc, seg.R);
  if (smem > 0 && seg.tab && seg.mask && !listed && Q >= 2 && mask_stride == 0 && tc.pair &&
      2 * smem <= (size_t)kTileOccSmemMax) {
    dim3 grid(tc.tiles_y * tc.tiles_z, (Q + 1) / 2);
    if (tc.pair == 2 && seg.tabw && tc.lanes == 32) {
      // rows without pad words: (TZ + 2R) (TY + 2R) wx words per query, one spare at each end
      const size_t smem_w = ((size_t)(tc.TZ + 2 * seg.R) * (tc.TY + 2 * seg.R) * d.wx + 2) * 8;
      if (counters)
        k_propagate_tile_pair<true, true><<<grid, 256, smem_w, st>>>(d, seg, tc, X, x_stride, mask, occ, out,
                                                                     out_stride, Q, xbox, obox, box_stride, counters);
      else
        k_propagate_tile_pair<false, true><<<grid, 256, smem_w, st>>>(d, seg, tc, X, x_stride, mask, occ, out,
                                                                      out_stride, Q, xbox, obox, box_stride,
                                                                      nullptr);
      return cudaGetLastError();
    }
    if (counters)
      k_propagate_tile_pair<true, false><<<grid, 256, 2 * smem, st>>>(d, seg, tc, X, x_stride, mask, occ, out,
                                                                      out_stride, Q, xbox, obox, box_stride,
                                                                      counters);
    else
      k_propagate_tile_pair<false, false><<<grid, 256, 2 * smem, st>>>(d, seg, tc, X, x_stride, mask, occ, out,
                                                                       out_stride, Q, xbox, obox, box_stride,
                                                                       nullptr);
    return cudaGetLastError();
  }
  if (smem > 0 && seg.tab && listed) {
    if (counters)
      k_propagate_tile_list<true><<<list_grid, 256, smem, st>>>(
          d, seg, tc, X, x_stride, mask, mask_stride, occ, out, out_stride, xbox, obox, box_stride, counters,
          wl->items, wl->count);
    else
      k_propagate_tile_list<false><<<list_grid, 256, smem, st>>>(
          d, seg, tc, X, x_stride, mask, mask_stride, occ, out, out_stride, xbox, obox, box_stride, nullptr,
          wl->items, wl->count);
    return cudaGetLastError();
  }
  if (smem > 0 && seg.tab) {
    dim3 grid(tc.tiles_y * tc.tiles_z, Q);
    if (counters)
      k_propagate_tile<true><<<grid, 256, smem, st>>>(d, seg, tc, X, x_stride, mask, mask_stride,
                                                             occ, out, out_stride, xbox, obox, box_stride,
                                                             counters);
    else
      k_propagate_tile<false><<<grid, 256, smem, st>>>(d, seg, tc, X, x_stride, mask, mask_stride,
                                                              occ, out, out_stride, xbox, obox, box_stride,
                                                              nullptr);
    return cudaGetLastError();
  }
  dim3 grid(grid_for(d.nw, 256), Q);
  if (counters)
    k_propagate<true><<<grid, 256, 0, st>>>(d, seg, X, x_stride, mask, mask_stride, occ, out,
                                            out_stride, xbox, obox, box_stride, counters);
  else
    k_propagate<false><<<grid, 256, 0, st>>>(d, seg, X, x_stride, mask, mask_stride, occ, out,
                                             out_stride, xbox, obox, box_stride, nullptr);
  return cudaGetLastError();
}

// --------------------------------------------------------------- seeds, and

__global__ void k_seed_points(Dims d, const int32_t* __restrict__ pts, const uint32_t* __restrict__ and_set,
                              const uint32_t* __restrict__ excl, uint32_t* __restrict__ out, long os,
                              const int32_t* __restrict__ gate, int32_t* __restrict__ obox, long bs) {
  const int q = blockIdx.y;
  const long w = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (w >= d.nw) return;
  uint32_t v = 0;
  const int x = pts[3 * q], y = pts[3 * q + 1], z = pts[3 * q + 2];
  if ((!gate || gate[q]) && inside(d, x, y, z)) {
    const long i = lin(d, x, y, z);
    if ((i >> 5) == w) v = 1u << (i & 31);
  }
  if (and_set) v &= __ldg(and_set + w);
  if (excl) v &= ~__ldg(excl + w);
  out[q * os + w] = v;
  if (v) {
    int32_t* b = obox + q * bs;
    atomicMin(b + 0, x >> 5);
    atomicMin(b + 1, y);
    atomicMin(b + 2, z);
    atomicMin(b + 3, -(x >> 5));
    atomicMin(b + 4, -y);
    atomicMin(b + 5, -z);
  }
}

cudaError_t launch_seed_points(const Dims& d, const int32_t* points, int Q, const uint32_t* and_set,
                               const uint32_t* excl, uint32_t* out, long out_stride,
                               const int32_t* found_gate, int32_t* obox, long box_stride,
                               cudaStream_t st) {
  if (Q <= 0) return cudaSuccess;
  dim3 grid(grid_for(d.nw, 256), Q);
  k_seed_points<<<grid, 256, 0, st>>>(d, points, and_set, excl, out, out_stride, found_gate, obox,
                                      box_stride);
  return cudaGetLastError();
}

__global__ void k_and(const uint32_t* __restrict__ a, const uint32_t* __restrict__ b, uint32_t* out,
                      long n) {
  const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i < n) out[i] = a[i] & b[i];
}

cudaError_t launch_and(const uint32_t* a, const uint32_t* b, uint32_t* out, long n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_and<<<grid_for(n, 256), 256, 0, st>>>(a, b, out, n);
  return cudaGetLastError();
}

// ----------------------------------------------------------- reach traceback

// One block per query.  p_0 = root; p_k = min linear index over the offsets
// e of segment k with q = p_{k-1} + e inside the grid, q in V_k and the
// segment p_{k-1} -> q free (edge-mask bit of p_{k-1} in row e).
// nearest != nullptr: minimise (|q - nearest_k|^2, index) instead.
__device__ void traceback_block(const Dims& d, const ArmDev& arm, int rx, int ry, int rz,
                                const uint32_t* V, const int32_t* nearest, int32_t* pose,
                                int32_t* found) {
  __shared__ unsigned long long best;
  __shared__ int p[3];
  __shared__ int ok;
  if (threadIdx.x == 0) {
    ok = inside(d, rx, ry, rz) && test_bit(V, lin(d, rx, ry, rz));
    p[0] = rx;
    p[1] = ry;
    p[2] = rz;
    *found = ok;
    pose[0] = ok ? rx : 0;
    pose[1] = ok ? ry : 0;
    pose[2] = ok ? rz : 0;
  }
  __syncthreads();
  if (!ok) {
    for (int i = threadIdx.x; i < 3 * arm.S; i += blockDim.x) pose[3 + i] = 0;
    return;
  }
  for (int k = 1; k <= arm.S; ++k) {
    const SegDev& sg = arm.seg[k - 1];
    const uint32_t* Vk = V + (long)k * d.nw;
    const int px = p[0], py = p[1], pz = p[2];
    const long pi = lin(d, px, py, pz);
    if (threadIdx.x == 0) best = ~0ull;
    __syncthreads();
    for (int e = threadIdx.x; e < sg.n; e += blockDim.x) {
      const int32_t o = __ldg(sg.off + e);
      const int qx = px + unpack_x(o), qy = py + unpack_y(o), qz = pz + unpack_z(o);
      if (!inside(d, qx, qy, qz)) continue;
      const long qi = lin(d, qx, qy, qz);
      if (!test_bit(Vk, qi)) continue;
      if (!edge_bit(d, sg, e, pi)) continue;
      unsigned long long key = (unsigned long long)qi;
      if (nearest) {
        const long dx = qx - nearest[3 * k], dy = qy - nearest[3 * k + 1], dz = qz - nearest[3 * k + 2];
        key |= (unsigned long long)(dx * dx + dy * dy + dz * dz) << 32;
      }
      atomicMin(&best, key);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      const long qi = (long)(best & 0xffffffffull);
      p[0] = (int)(qi % d.nx);
      p[1] = (int)((qi / d.nx) % d.ny);
      p[2] = (int)(qi / ((long)d.nx * d.ny));
      pose[3 * k] = p[0];
      pose[3 * k + 1] = p[1];
      pose[3 * k + 2] = p[2];
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(256) k_traceback(Dims d, ArmDev arm, const int32_t* __restrict__ root,
                                                   const uint32_t* __restrict__ V, long vs,
                                                   int32_t* poses, int32_t* found) {
  const int q = blockIdx.x;
  traceback_block(d, arm, root[0], root[1], root[2], V + q * vs, nullptr,
                  poses + (long)q * 3 * (arm.S + 1), found + q);
}

cudaError_t launch_traceback(const Dims& d, const ArmDev& arm, const int32_t* root, const uint32_t* V,
                             long vstride, int Q, int32_t* poses, int32_t* found, cudaStream_t st) {
  if (Q <= 0) return cudaSuccess;
  k_traceback<<<Q, 256, 0, st>>>(d, arm, root, V, vstride, poses, found);
  return cudaGetLastError();
}

// Batched re-solve of reach poses (replan): block q handles slot q when
// gate[q] is set, minimising (squared distance to old pose, index).
__global__ void __launch_bounds__(256) k_traceback_nearest(Dims d, ArmDev arm, const int32_t* root,
                                                           const uint32_t* V, long vs,
                                                           const int32_t* old_pose, long ops,
                                                           int32_t* pose, int32_t* found,
                                                           const int32_t* gate) {
  const int q = blockIdx.x;
  if (gate && !gate[q]) return;
  traceback_block(d, arm, root[0], root[1], root[2], V + q * vs, old_pose + q * ops,
                  pose + (long)q * 3 * (arm.S + 1), found + q);
}

cudaError_t launch_traceback_nearest(const Dims& d, const ArmDev& arm, const int32_t* root,
                                     const uint32_t* V, const int32_t* old_pose, int32_t* pose,
                                     int32_t* found, cudaStream_t st) {
  k_traceback_nearest<<<1, 256, 0, st>>>(d, arm, root, V, 0, old_pose, 0, pose, found, nullptr);
  return cudaGetLastError();
}

cudaError_t launch_traceback_nearest_many(const Dims& d, const ArmDev& arm, const int32_t* root,
                                          const uint32_t* V, long vstride, const int32_t* old_pose,
                                          long old_stride, int32_t* pose, int32_t* found,
                                          const int32_t* gate, int Q, cudaStream_t st) {
  if (Q <= 0) return cudaSuccess;
  k_traceback_nearest<<<Q, 256, 0, st>>>(d, arm, root, V, vstride, old_pose, old_stride, pose, found,
                                          gate);
  return cudaGetLastError();
}

// --------------------------------------------------------- batched replan

// Per slot r (c[r] in [0, W) marks a live slot): cut = some pose after c is
// invalid now; need = cut and the reach pose itself is invalid (re-solve it
// from its end effector, tgt[r]); the slot's relaxation record is zeroed.
__global__ void k_replan_prepare(int W, int S, const int32_t* __restrict__ poses_in,
                                 const int32_t* __restrict__ c, const int32_t* __restrict__ valid,
                                 int32_t* cut, int32_t* need, int32_t* tgt, int32_t* relax) {
  const int r = blockIdx.x;
  const int cr = c[r];
  const bool live = cr >= 0 && cr < W;
  for (int i = threadIdx.x; i < 2 * W; i += blockDim.x) relax[(long)r * 2 * W + i] = 0;
  if (threadIdx.x != 0) return;
  int k = 0;
  if (live)
    for (int j = cr + 1; j < W; ++j)
      if (!valid[(long)r * W + j]) k = 1;
  const int n = k && !valid[(long)r * W + W - 1];
  cut[r] = k;
  need[r] = n;
  const int32_t* end = poses_in + (((long)r * W + W - 1) * (S + 1) + S) * 3;
  tgt[3 * r] = n ? end[0] : -1;
  tgt[3 * r + 1] = n ? end[1] : -1;
  tgt[3 * r + 2] = n ? end[2] : -1;
}

// Cut slots whose reach pose is still valid keep it; gate = cut and a reach
// pose exists (re-solved or kept).
__global__ void k_replan_fix(int W, int S, const int32_t* __restrict__ poses_in,
                             const int32_t* __restrict__ cut, const int32_t* __restrict__ need,
                             int32_t* reach, int32_t* rfound, int32_t* gate) {
  const int r = blockIdx.x;
  const long ps = 3L * (S + 1);
  if (cut[r] && !need[r]) {
    for (int i = threadIdx.x; i < ps; i += blockDim.x)
      reach[r * ps + i] = poses_in[((long)r * W + W - 1) * ps + i];
    if (threadIdx.x == 0) rfound[r] = 1;
  }
  __syncthreads();
  if (threadIdx.x == 0) gate[r] = cut[r] && (need[r] ? rfound[r] : 1);
}

// Statuses of the slots the smooth chain does not run: live and uncut =
// kept (poses already copied); cut without a reach pose = unreachable, the
// poses after c repeat pose c with m = -1.
__global__ void k_replan_finalize(int W, int S, const int32_t* __restrict__ c,
                                  const int32_t* __restrict__ cut, const int32_t* __restrict__ gate,
                                  int32_t* poses, int32_t* relax, int32_t* status) {
  const int r = blockIdx.x;
  const int cr = c[r];
  if (cr < 0 || cr >= W || gate[r]) return;
  const long ps = 3L * (S + 1);
  if (!cut[r]) {
    if (threadIdx.x == 0) status[r] = IK_PATH_KEPT;
    return;
  }
  for (int j = cr + 1; j < W; ++j) {
    for (int i = threadIdx.x; i < ps; i += blockDim.x)
      poses[((long)r * W + j) * ps + i] = poses[((long)r * W + cr) * ps + i];
    if (threadIdx.x == 0) relax[((long)r * W + j) * 2] = -1;
  }
  if (threadIdx.x == 0) status[r] = IK_PATH_UNREACHABLE;
}

cudaError_t launch_replan_prepare(int R, int W, int S, const int32_t* poses_in, const int32_t* c,
                                  const int32_t* valid, int32_t* cut, int32_t* need, int32_t* tgt,
                                  int32_t* relax, cudaStream_t st) {
  if (R <= 0) return cudaSuccess;
  k_replan_prepare<<<R, 64, 0, st>>>(W, S, poses_in, c, valid, cut, need, tgt, relax);
  return cudaGetLastError();
}

cudaError_t launch_replan_fix(int R, int W, int S, const int32_t* poses_in, const int32_t* cut,
                              const int32_t* need, int32_t* reach, int32_t* rfound, int32_t* gate,
                              cudaStream_t st) {
  if (R <= 0) return cudaSuccess;
  k_replan_fix<<<R, 64, 0, st>>>(W, S, poses_in, cut, need, reach, rfound, gate);
  return cudaGetLastError();
}

cudaError_t launch_replan_finalize(int R, int W, int S, const int32_t* c, const int32_t* cut,
                                   const int32_t* gate, int32_t* poses, int32_t* relax,
                                   int32_t* status, cudaStream_t st) {
  if (R <= 0) return cudaSuccess;
  k_replan_finalize<<<R, 64, 0, st>>>(W, S, c, cut, gate, poses, relax, status);
  return cudaGetLastError();
}

// ------------------------------------------------------------ validate poses

// Shell index of offset (x, y, z) in device order (row (z, y), then a scan
// of the row's x offsets); -1 when the offset is not in the shell.
__device__ int shell_index(const SegDev& sg, int x, int y, int z) {
  const int n2 = x * x + y * y + z * z;
  if (n2 < sg.lo2 || n2 > sg.hi2) return -1;
  if (y < -sg.R || y > sg.R || z < -sg.R || z > sg.R) return -1;
  const int r = (z + sg.R) * (2 * sg.R + 1) + (y + sg.R);
  const int r1 = __ldg(sg.rows + r + 1);
  for (int e = __ldg(sg.rows + r); e < r1; ++e)
    if (unpack_x(__ldg(sg.off + e)) == x) return e;
  return -1;
}

// One thread per (pose, segment); valid[pose] starts at 1 and is cleared by
// any segment that leaves the grid, leaves its shell or meets an obstacle.
__global__ void k_validate(Dims d, ArmDev arm, const uint32_t* __restrict__ occ,
                           const int32_t* __restrict__ poses, int n, int32_t* valid) {
  const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (t >= (long)n * arm.S) return;
  const int i = (int)(t / arm.S), k = (int)(t % arm.S) + 1;
  const int32_t* P = poses + (long)i * 3 * (arm.S + 1);
  const int ax = P[3 * (k - 1)], ay = P[3 * (k - 1) + 1], az = P[3 * (k - 1) + 2];
  const int bx = P[3 * k], by = P[3 * k + 1], bz = P[3 * k + 2];
  bool ok = inside(d, ax, ay, az) && inside(d, bx, by, bz);
  if (ok) {
    const SegDev& sg = arm.seg[k - 1];
    const int e = shell_index(sg, bx - ax, by - ay, bz - az);
    ok = e >= 0;
    if (ok) {
      const int s0 = __ldg(sg.sc_start + e), s1 = __ldg(sg.sc_start + e + 1);
      for (int j = s0; j < s1 && ok; ++j) {
        const int32_t v = __ldg(sg.sc + j);
        ok = !test_bit(occ, lin(d, ax + unpack_x(v), ay + unpack_y(v), az + unpack_z(v)));
      }
    }
  }
  if (!ok) atomicAnd(valid + i, 0);
}

__global__ void k_seed_set(Dims d, const uint32_t* __restrict__ T, const uint32_t* __restrict__ F,
                           uint32_t* __restrict__ out, int32_t* __restrict__ obox) {
  const long w = blockIdx.x * (long)blockDim.x + threadIdx.x;
  uint32_t v = 0;
  int wx = 0, y = 0, z = 0;
  if (w < d.nw) {
    word_coords(d, w, &wx, &y, &z);
    v = __ldg(T + w) & __ldg(F + w);
    out[w] = v;
  }
  box_accumulate(obox, v != 0, wx, y, z);
}

cudaError_t launch_seed_set(const Dims& d, const uint32_t* T, const uint32_t* F, uint32_t* out,
                            int32_t* obox, cudaStream_t st) {
  k_seed_set<<<grid_for(d.nw, 256), 256, 0, st>>>(d, T, F, out, obox);
  return cudaGetLastError();
}

__global__ void k_fill_i32(int32_t* p, long n, int32_t v) {
  const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

cudaError_t launch_fill_i32(int32_t* p, long n, int32_t v, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_fill_i32<<<grid_for(n, 256), 256, 0, st>>>(p, n, v);
  return cudaGetLastError();
}

cudaError_t launch_validate(const Dims& d, const ArmDev& arm, const uint32_t* occ,
                            const int32_t* poses, int n, int32_t* valid, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_fill_i32<<<grid_for(n, 256), 256, 0, st>>>(valid, n, 1);
  const long t = (long)n * arm.S;
  k_validate<<<grid_for(t, 256), 256, 0, st>>>(d, arm, occ, poses, n, valid);
  return cudaGetLastError();
}

// ------------------------------------------------ guide points + targets

// Adds voxel (x, y, z) to a min-form word box.
__device__ __forceinline__ void box_point(int32_t* b, int x, int y, int z) {
  atomicMin(b + 0, x >> 5);
  atomicMin(b + 1, y);
  atomicMin(b + 2, z);
  atomicMin(b + 3, -(x >> 5));
  atomicMin(b + 4, -y);
  atomicMin(b + 5, -z);
}

__device__ __forceinline__ long floor_div(long a, long b) {  // b > 0
  long q = a / b;
  if ((a % b != 0) && (a < 0)) --q;
  return q;
}

__device__ __forceinline__ int isqrt_dev(int v) {  // floor(sqrt(v)), v >= 0
  int r = (int)sqrtf((float)v);
  while (r * r > v) --r;
  while ((r + 1) * (r + 1) <= v) ++r;
  return r;
}

// One block per (path, waypoint).  Guide point by the nominal-arc rule, then
// the waypoint target set T_j (free voxels within squared distance eps2,
// grown to eps2_max when empty; T_{W-1} = {end effector}) intersected with
// F_S, OR-ed into the (pre-zeroed) last survivor set of the waypoint.
// Guide point and waypoint target of waypoint j of path p (one block).
__device__ void guide_targets_block(const Dims& d, const ArmDev& arm, const GuideArm& ga,
                                    const uint32_t* __restrict__ occ, const uint32_t* __restrict__ F_S,
                                    const int32_t* __restrict__ reach, const int32_t* __restrict__ found,
                                    int W, int eps2, int eps2_max, int32_t* g, int32_t* eps_used,
                                    uint32_t* Vw, int32_t* wbox, const int32_t* __restrict__ c_arr,
                                    int32_t* __restrict__ fold_at, int p, int j) {
  if (c_arr && j <= c_arr[p]) return;  // replan: waypoints up to the current one stay
  const int S = arm.S;    // layout of the waypoint sets
  const int GS = ga.S;    // the guide polyline's segments
  const int32_t* R = reach + (long)p * 3 * (ga.pose_joints > 0 ? ga.pose_joints : GS + 1);
  __shared__ int gp[3];
  __shared__ int used;
  const bool ok = !found || found[p];
  if (threadIdx.x == 0 && ga.n_per_seg > 0) {
    // n points per segment: the i-th of segment k at p_{k-1} + (i/n)(p_k -
    // p_{k-1}), rounded half up, and the last one at p_GS
    const int n = ga.n_per_seg;
    int k = j / n + 1, i = j - (k - 1) * n;
    if (k > GS) {
      k = GS;
      i = n;
    }
    for (int c = 0; c < 3; ++c) {
      const long a = ok ? R[3 * (k - 1) + c] : 0, b = ok ? R[3 * k + c] : 0;
      gp[c] = (int)(a + floor_div(2L * i * (b - a) + n, 2L * n));
      g[((long)p * W + j) * 3 + c] = gp[c];
    }
    if (fold_at && ga.fold_len > 0) {
      // n times the arc length fold_len beyond this guide point, and the
      // segment of the polyline (the fold segment GS + 1 included) it lands on
      long C = 0;
      for (int q = 0; q < k - 1; ++q) C += ga.len[q];
      const long T = (long)n * C + (long)i * ga.len[k - 1] + (long)n * ga.fold_len;
      // segment kk with n C_{kk-1} <= T < n C_kk; the fold segment when T
      // is its far end
      int kk = GS + 1;
      long c0 = 0, run = 0;
      for (int q = 1; q <= GS + 1; ++q) {
        const long lq = q <= GS ? ga.len[q - 1] : ga.fold_len;
        if ((long)n * run <= T && T < (long)n * (run + lq)) {
          kk = q;
          break;
        }
        run += lq;
      }
      if (kk == GS + 1) {
        c0 = 0;
        for (int q = 0; q < GS; ++q) c0 += ga.len[q];
      } else {
        c0 = run;
      }
      const long lk = kk <= GS ? ga.len[kk - 1] : ga.fold_len;
      const long den = (long)n * lk, num = T - (long)n * c0;
      int32_t* fa = fold_at + ((long)p * W + j) * 4;
      for (int c = 0; c < 3; ++c) {
        const long a = ok ? R[3 * (kk - 1) + c] : 0, b = ok ? R[3 * kk + c] : 0;
        fa[c] = (int32_t)(den * a + num * (b - a));
      }
      fa[3] = (int32_t)den;
    }
    used = -1;
  } else if (threadIdx.x == 0) {
    long lam = 0;
    for (int k = 0; k < GS; ++k) lam += ga.len[k];
    const long num = (long)j * lam;
    long Cprev = 0;
    int k = GS;
    long c0 = 0;
    for (int kk = 1; kk <= GS; ++kk) {
      const long c1 = Cprev + ga.len[kk - 1];
      if (Cprev * (W - 1) <= num && num < c1 * (W - 1)) {
        k = kk;
        c0 = Cprev;
        break;
      }
      Cprev = c1;
    }
    if (k == GS) c0 = lam - ga.len[GS - 1];
    const long r = num - c0 * (W - 1);
    const long den = (long)ga.len[k - 1] * (W - 1);
    for (int i = 0; i < 3; ++i) {
      const long a = ok ? R[3 * (k - 1) + i] : 0, b = ok ? R[3 * k + i] : 0;
      gp[i] = (int)(a + floor_div(2 * r * (b - a) + den, 2 * den));
      g[((long)p * W + j) * 3 + i] = gp[i];
    }
    used = -1;
  }
  __syncthreads();
  if (!Vw) return;  // guide points only
  uint32_t* VS = Vw + (((long)p * W + j) * (S + 1) + S) * d.nw;
  int32_t* vb = wbox + (((long)p * W + j) * (S + 1) + S) * 6;
  if (!ok) {
    if (threadIdx.x == 0) eps_used[(long)p * W + j] = -1;
    return;
  }
  if (j == W - 1) {
    if (threadIdx.x == 0) {
      const int tx = R[3 * GS], ty = R[3 * GS + 1], tz = R[3 * GS + 2];
      if (inside(d, tx, ty, tz)) {
        const long i = lin(d, tx, ty, tz);
        if (test_bit(F_S, i)) {
          atomicOr(VS + (i >> 5), 1u << (i & 31));
          box_point(vb, tx, ty, tz);
        }
      }
      eps_used[(long)p * W + j] = 0;
    }
    return;
  }
  const int top = max(eps2, eps2_max);
  for (int e2 = eps2; e2 <= top; ++e2) {
    const int Rb = isqrt_dev(e2);
    const int side = 2 * Rb + 1;
    int any = 0;
    for (int t = threadIdx.x; t < side * side * side; t += blockDim.x) {
      const int x = gp[0] - Rb + t % side, y = gp[1] - Rb + (t / side) % side,
                z = gp[2] - Rb + t / (side * side);
      const int dx = x - gp[0], dy = y - gp[1], dz = z - gp[2];
      if (dx * dx + dy * dy + dz * dz > e2 || !inside(d, x, y, z)) continue;
      if (!test_bit(occ, lin(d, x, y, z))) any = 1;
    }
    if (__syncthreads_or(any)) {
      if (threadIdx.x == 0) used = e2;
      break;
    }
  }
  __syncthreads();
  const int e2 = used;
  if (threadIdx.x == 0) eps_used[(long)p * W + j] = e2;
  if (e2 < 0) return;
  const int Rb = isqrt_dev(e2);
  const int side = 2 * Rb + 1;
  for (int t = threadIdx.x; t < side * side * side; t += blockDim.x) {
    const int x = gp[0] - Rb + t % side, y = gp[1] - Rb + (t / side) % side,
              z = gp[2] - Rb + t / (side * side);
    const int dx = x - gp[0], dy = y - gp[1], dz = z - gp[2];
    if (dx * dx + dy * dy + dz * dz > e2 || !inside(d, x, y, z)) continue;
    const long i = lin(d, x, y, z);
    if (!test_bit(occ, i) && test_bit(F_S, i)) {
      atomicOr(VS + (i >> 5), 1u << (i & 31));
      box_point(vb, x, y, z);
    }
  }
}

__global__ void k_guide_targets(Dims d, ArmDev arm, GuideArm ga, const uint32_t* __restrict__ occ,
                                const uint32_t* __restrict__ F_S, const int32_t* __restrict__ reach,
                                const int32_t* __restrict__ found, int W, int j_lo, int eps2,
                                int eps2_max, int32_t* g, int32_t* eps_used, uint32_t* Vw,
                                int32_t* wbox, const int32_t* __restrict__ c_arr,
                                int32_t* __restrict__ fold_at) {
  guide_targets_block(d, arm, ga, occ, F_S, reach, found, W, eps2, eps2_max, g, eps_used, Vw, wbox, c_arr,
                      fold_at, blockIdx.y, blockIdx.x + j_lo);
}

cudaError_t launch_guide_targets(const Dims& d, const ArmDev& arm, const uint32_t* occ,
                                 const uint32_t* F_S, const int32_t* reach, const int32_t* found,
                                 int P, int W, int j_lo, int eps2, int eps2_max, int32_t* g,
                                 int32_t* eps_used, uint32_t* Vw, int32_t* wbox, cudaStream_t st,
                                 const int32_t* c_arr, const GuideArm* ga, int32_t* fold_at) {
  if (P <= 0 || W - j_lo <= 0) return cudaSuccess;
  GuideArm own;
  if (!ga) {
    own.S = arm.S;
    for (int k = 0; k < arm.S; ++k) own.len[k] = arm.len[k];
    ga = &own;
  }
  dim3 grid(W - j_lo, P);
  k_guide_targets<<<grid, 128, 0, st>>>(d, arm, *ga, occ, F_S, reach, found, W, j_lo, eps2, eps2_max, g,
                                        eps_used, Vw, wbox, c_arr, fold_at);
  return cudaGetLastError();
}

// ----------------------------------------------------- smooth chain per path

// Sets written earlier in the same kernel are read with plain loads (the
// read-only path is not coherent with in-kernel writes).
__device__ __forceinline__ uint32_t ld_shifted_rw(const uint32_t* s, const Dims& d, int wx, int y, int z,
                                                  int dx, int dy, int dz) {
  const int yy = y + dy, zz = z + dz;
  if ((unsigned)yy >= (unsigned)d.ny || (unsigned)zz >= (unsigned)d.nz) return 0u;
  const uint32_t* row = s + ((long)zz * d.ny + yy) * d.wx;
  const int w0 = wx + (dx >> 5);
  const int sh = dx & 31;
  const uint32_t lo = ((unsigned)w0 < (unsigned)d.wx) ? row[w0] : 0u;
  if (sh == 0) return lo;
  const uint32_t hi = ((unsigned)(w0 + 1) < (unsigned)d.wx) ? row[w0 + 1] : 0u;
  return __funnelshift_r(lo, hi, sh);
}

// Bits of word (wx, y, z) inside the ball |v - c|^2 <= d2.
__device__ __forceinline__ uint32_t ball_bits(int wx, int y, int z, const int* c, int d2) {
  const int dy = y - c[1], dz = z - c[2];
  const int rem = d2 - dy * dy - dz * dz;
  if (rem < 0) return 0u;
  const int r = isqrt_dev(rem);
  const int lo = max(c[0] - r, 32 * wx) - 32 * wx, hi = min(c[0] + r, 32 * wx + 31) - 32 * wx;
  if (lo > hi) return 0u;
  const uint32_t upto = hi == 31 ? 0xffffffffu : ((1u << (hi + 1)) - 1u);
  return upto & ~((1u << lo) - 1u);
}

struct Box {
  int x0, x1, y0, y1, z0, z1;  // inclusive voxel ranges, clipped to the grid
};

constexpr int kChainThreads = 512;


struct ChainShared {
  int ref[IK_MAX_SEG + 1][3];
  Box box[IK_MAX_SEG + 1];
  int r2[IK_MAX_SEG + 1];  // squared ball radius of joint k, -1: no ball
  int empty;               // some joint's search box is empty
  unsigned long long best;
  int cur[3];
  unsigned long long* cnt;  // work counters (ChainArgs::counters), nullable
};

// Search boxes of one feasibility test at relaxation m: the root voxel for
// joint 0; for a filtered joint k the box of Ball(ref_k, rad[k] + m); for an
// unfiltered one the box of its survivor set (vb: the S + 1 min-form word
// boxes of this waypoint's sets).
__device__ void chain_boxes(const Dims& d, ChainShared& sh, int S, int m, const int* rad,
                            const int32_t* vb) {
  if (threadIdx.x == 0) sh.empty = 0;
  __syncthreads();
  if (threadIdx.x <= S) {
    const int k = threadIdx.x;
    Box b;
    if (k == 0) {
      b = Box{sh.ref[0][0], sh.ref[0][0], sh.ref[0][1], sh.ref[0][1], sh.ref[0][2], sh.ref[0][2]};
      sh.r2[0] = -1;
    } else if (rad[k] >= 0) {
      const int r = rad[k] + m;
      b.x0 = max(0, sh.ref[k][0] - r);
      b.x1 = min(d.nx - 1, sh.ref[k][0] + r);
      b.y0 = max(0, sh.ref[k][1] - r);
      b.y1 = min(d.ny - 1, sh.ref[k][1] + r);
      b.z0 = max(0, sh.ref[k][2] - r);
      b.z1 = min(d.nz - 1, sh.ref[k][2] + r);
      sh.r2[k] = r * r;
    } else {
      const int32_t* v = vb + 6 * k;
      const int wx0 = v[0], wx1 = -v[3];
      if (wx0 > wx1) {
        b = Box{0, -1, 0, -1, 0, -1};
        sh.empty = 1;
      } else {
        b = Box{32 * wx0, min(d.nx - 1, 32 * wx1 + 31), v[1], -v[4], v[2], -v[5]};
      }
      sh.r2[k] = -1;
    }
    sh.box[k] = b;
  }
  __syncthreads();
}

// Number of words of a box and the coordinates of its t-th word.
__device__ __forceinline__ long box_words(const Box& b) {
  return (long)((b.x1 >> 5) - (b.x0 >> 5) + 1) * (b.y1 - b.y0 + 1) * (b.z1 - b.z0 + 1);
}
__device__ __forceinline__ void box_word(const Box& b, long t, int* wx, int* y, int* z) {
  const int nwx = (b.x1 >> 5) - (b.x0 >> 5) + 1, ny = b.y1 - b.y0 + 1;
  *wx = (b.x0 >> 5) + (int)(t % nwx);
  *y = b.y0 + (int)((t / nwx) % ny);
  *z = b.z0 + (int)(t / ((long)nwx * ny));
}

__device__ void chain_clear(const Dims& d, ChainShared& sh, int S, uint32_t* R, uint32_t* U) {
  for (int k = 0; k <= S; ++k) {
    const Box b = sh.box[k];
    const long n = box_words(b);
    for (long t = threadIdx.x; t < n; t += blockDim.x) {
      int wx, y, z;
      box_word(b, t, &wx, &y, &z);
      const long w = ((long)z * d.ny + y) * d.wx + wx;
      R[(long)k * d.nw + w] = 0u;
      U[(long)k * d.nw + w] = 0u;
    }
  }
  __syncthreads();
}

// Occupancy of the box that holds every supercover voxel one level of the
// chain can test, staged in shared memory: a segment runs from a voxel of
// one box to a voxel of the other, so its supercover lies in the hull of the
// two boxes (one extra word on either side in x, read by the funnel shifts
// for bits that the result masks away).  Larger boxes (strong relaxation)
// keep reading the occupancy in global memory: staging a big hull at every
// level costs more than the L2-resident reads it replaces (measured).  The
// level's source set, which lies in its own ball box, is staged the same way
// (with the extra word on either side).  Both live in the kernel's dynamic
// shared memory: kChainOccWords words for the occupancy, then kChainSrcWords
// for the source.
constexpr int kChainOccWords = 10240;
constexpr int kChainSrcWords = 8192;

// A box of words staged in shared memory: words w0 .. w0 + nw - 1 of rows
// y0 .. y0 + ny - 1 of slices z0 ..; ok = false when it did not fit.
struct OccBox {
  const uint32_t* s;
  int w0, y0, z0, nw, ny;
  bool ok;
};

__device__ __forceinline__ OccBox word_box(const Box& a, const Box& b, uint32_t* s, int cap, int* nz,
                                           long* total) {
  OccBox ob;
  ob.s = s;
  ob.w0 = (min(a.x0, b.x0) >> 5) - 1;
  ob.y0 = min(a.y0, b.y0);
  ob.z0 = min(a.z0, b.z0);
  ob.nw = (max(a.x1, b.x1) >> 5) + 1 - ob.w0 + 1;
  ob.ny = max(a.y1, b.y1) - ob.y0 + 1;
  *nz = max(a.z1, b.z1) - ob.z0 + 1;
  *total = (long)ob.nw * ob.ny * *nz;
  ob.ok = *total <= cap;
  return ob;
}

// The offset table and row starts a level's restricted words read: the
// segment's own (global memory), or, with stored edge masks (the occupancy
// buffer then free), the planes the level can use staged in shared memory,
// so that the walk's table reads do not go to L2 behind the mask loads.
// off[e] and rows[r] are valid for the staged e and r (plain loads).
struct ChainTab {
  const int32_t* off;
  const int32_t* rows;
};

// Stages, for one level, the occupancy of the hull of boxes a and b and the
// source set `src` (written earlier in this kernel: plain loads) over box sb;
// with tab, the table (see ChainTab) for outputs in a and sources in sb.
__device__ void chain_stage(const Dims& d, const SegDev& sg, const Box& a, const Box& b, const Box& sb,
                            const uint32_t* src, uint32_t* so, OccBox* ob, OccBox* xb,
                            ChainTab* tab = nullptr) {
  int nz_o, nz_x;
  long tot_o, tot_x;
  // with stored edge masks one mask word per test beats a walk: no occupancy
  *ob = word_box(a, b, so, sg.mask ? -1 : kChainOccWords, &nz_o, &tot_o);
  *xb = word_box(sb, sb, so + kChainOccWords, src ? kChainSrcWords : -1, &nz_x, &tot_x);
  __syncthreads();  // the previous level's readers are done with the buffers
  if (ob->ok) {
    uint32_t* s = so;
    for (int t = threadIdx.x; t < tot_o; t += blockDim.x) {
      const int ww = ob->w0 + t % ob->nw, yy = ob->y0 + (t / ob->nw) % ob->ny, zz = ob->z0 + t / (ob->nw * ob->ny);
      s[t] = (ww >= 0 && ww < d.wx) ? __ldg(sg.occ + ((long)zz * d.ny + yy) * d.wx + ww) : 0u;
    }
  }
  if (xb->ok) {
    uint32_t* s = so + kChainOccWords;
    for (int t = threadIdx.x; t < tot_x; t += blockDim.x) {
      const int ww = xb->w0 + t % xb->nw, yy = xb->y0 + (t / xb->nw) % xb->ny, zz = xb->z0 + t / (xb->nw * xb->ny);
      s[t] = (ww >= 0 && ww < d.wx) ? src[((long)zz * d.ny + yy) * d.wx + ww] : 0u;
    }
  }
  if (tab) {
    tab->off = sg.off;
    tab->rows = sg.rows;
    const int R = sg.R, side = 2 * R + 1;
    const int pz0 = max(sb.z0 - a.z1, -R), pz1 = min(sb.z1 - a.z0, R);
    if (sg.mask && !ob->ok && pz0 <= pz1) {
      // rows of planes pz0 .. pz1 (and the end of the last), their offsets
      const int r0 = (pz0 + R) * side, nr = (pz1 - pz0 + 1) * side + 1;
      const int e0 = __ldg(sg.rows + r0), ne = __ldg(sg.rows + r0 + nr - 1) - e0;
      if (nr + ne <= kChainOccWords) {
        int32_t* s = reinterpret_cast<int32_t*>(so);
        for (int t = threadIdx.x; t < nr; t += blockDim.x) s[t] = __ldg(sg.rows + r0 + t);
        for (int t = threadIdx.x; t < ne; t += blockDim.x) s[nr + t] = __ldg(sg.off + e0 + t);
        tab->rows = s - r0;
        tab->off = s + nr - e0;
      }
    }
  }
  __syncthreads();
}

__device__ OccBox chain_stage_occ(const Dims& d, const SegDev& sg, const Box& a, const Box& b,
                                  uint32_t* s) {
  OccBox ob, xb;
  chain_stage(d, sg, a, b, a, nullptr, s, &ob, &xb);
  return ob;
}

// edge_word with the supercover walked against a staged occupancy box
__device__ __forceinline__ uint32_t edge_word_box(const Dims& d, const SegDev& sg, const OccBox& ob, int e,
                                                  long w, int wx, int y, int z) {
  if (!ob.ok) return edge_word(d, sg, e, w, wx, y, z);
  const int s1 = __ldg(sg.sc_start + e + 1);
  const uint32_t* base = ob.s + ((z - ob.z0) * ob.ny + (y - ob.y0)) * ob.nw + (wx - ob.w0);
  auto voxel = [&](int i) {
    const int32_t v = __ldg(sg.sc + i);
    const int vx = unpack_x(v);
    const uint32_t* row = base + (unpack_z(v) * ob.ny + unpack_y(v)) * ob.nw + (vx >> 5);
    return __funnelshift_r(row[0], row[1], vx);  // shift taken mod 32
  };
  uint32_t blocked = 0;
  int i = __ldg(sg.sc_start + e);
  // four independent reads per pass, the all-blocked exit checked per pass
  for (; i + 4 <= s1 && blocked != 0xffffffffu; i += 4)
    blocked |= voxel(i) | voxel(i + 1) | voxel(i + 2) | voxel(i + 3);
  for (; i < s1; ++i) blocked |= voxel(i);
  return ~blocked;
}

// One restricted propagation word: OR over the segment's offsets of the
// source set shifted by the offset, limited to offsets whose source voxels
// can fall in the source box, AND edge mask, within `m`.
// One restricted propagation word, its offset walk shared by the kG lanes
// of a lane group (lane g of the group takes every kG-th offset of each
// row run); the group's partial results are OR-reduced.  Sources are limited
// to offsets whose source voxels can fall in the source box.  Every lane of
// the group must call it (idle lanes pass m = 0).
constexpr int kG = 8;

__device__ __forceinline__ uint32_t restricted_word(const Dims& d, const SegDev& sg, const ChainTab& tab,
                                                    const OccBox& ob, const OccBox& xb, const uint32_t* src,
                                                    const Box& sb, int wx, int y, int z, long w, uint32_t m,
                                                    unsigned long long* cnt) {
  const int g = threadIdx.x % kG;
  const unsigned gmask = ((1u << kG) - 1u) << ((threadIdx.x & 31) & ~(kG - 1));
  uint32_t acc = 0;
  unsigned long long visited = 0, nonzero = 0;
  if (m) {
    const int R = sg.R, side = 2 * R + 1;
    const int ez0 = max(sb.z0 - z, -R), ez1 = min(sb.z1 - z, R);
    const int ey0 = max(sb.y0 - y, -R), ey1 = min(sb.y1 - y, R);
    const int exlo = sb.x0 - 32 * wx - 31, exhi = sb.x1 - 32 * wx;
    // the source word of an offset (0 when its voxels cannot lie in sb)
    auto source = [&](int e, int ez) -> uint32_t {
      const int32_t o = tab.off[e];
      const int ex = unpack_x(o);
      if (ex < exlo || ex > exhi) return 0u;
      if (xb.ok) {
        const uint32_t* row = xb.s + ((z + ez - xb.z0) * xb.ny + (y + unpack_y(o) - xb.y0)) * xb.nw +
                              (wx + (ex >> 5) - xb.w0);
        return __funnelshift_r(row[0], row[1], ex);  // shift taken mod 32
      }
      return ld_shifted_rw(src, d, wx, y, z, ex, unpack_y(o), ez);
    };
    for (int ez = ez0; ez <= ez1 && ey0 <= ey1; ++ez) {
      const int32_t* rowp = tab.rows + (ez + R) * side + R;
      const int e1 = rowp[ey1 + 1];
      for (int e = rowp[ey0] + g; e < e1; e += kG) {
        const uint32_t x = source(e, ez);
        if (cnt) {
          ++visited;
          nonzero += x != 0u;
        }
        if (x & m & ~acc) acc |= x & edge_word_box(d, sg, ob, e, w, wx, y, z);
      }
    }
  }
  if (cnt && visited) {
    atomicAdd(cnt + 0, visited);
    atomicAdd(cnt + 1, nonzero);
  }
  return __reduce_or_sync(gmask, acc) & m;
}

// Forward restriction: R_0 = {root}, R_k = (V_k & Ball(ref_k, r_k)) & D_k(R_{k-1})
// (no ball for an unfiltered joint).
__device__ bool chain_forward(const Dims& d, const ArmDev& arm, ChainShared& sh, const uint32_t* V,
                              uint32_t* R, uint32_t* so) {
  const int S = arm.S;
  if (threadIdx.x == 0) {
    const long i = lin(d, sh.ref[0][0], sh.ref[0][1], sh.ref[0][2]);
    R[i >> 5] = 1u << (i & 31);
  }
  __syncthreads();
  for (int k = 1; k <= S; ++k) {
    const Box b = sh.box[k], sb = sh.box[k - 1];
    const SegDev& sg = arm.segf[k - 1];  // the forward gather reads the mirrored offsets
    const uint32_t* src = R + (long)(k - 1) * d.nw;
    const uint32_t* Vk = V + (long)k * d.nw;
    uint32_t* dst = R + (long)k * d.nw;
    const long n = box_words(b);
    OccBox ob, xb;
    ChainTab tab;
    chain_stage(d, sg, b, sb, sb, src, so, &ob, &xb, &tab);
    int any = 0;
    // kG lanes per word; the loop bound is uniform per lane group
    for (long t0 = 0; t0 < n; t0 += blockDim.x / kG) {
      const long t = t0 + threadIdx.x / kG;
      int wx = 0, y = 0, z = 0;
      long w = 0;
      uint32_t m = 0;
      if (t < n) {
        box_word(b, t, &wx, &y, &z);
        w = ((long)z * d.ny + y) * d.wx + wx;
        m = (sh.r2[k] >= 0 ? ball_bits(wx, y, z, sh.ref[k], sh.r2[k]) : 0xffffffffu) & __ldg(Vk + w);
      }
      const uint32_t acc = restricted_word(d, sg, tab, ob, xb, src, sb, wx, y, z, w, m, sh.cnt);
      if (acc && threadIdx.x % kG == 0) {
        dst[w] = acc;
        any = 1;
      }
    }
    if (!__syncthreads_or(any)) return false;
  }
  return true;
}

// Backward restriction: U_S = R_S, U_k = R_k & D_{k+1}(U_{k+1}).
__device__ void chain_backward(const Dims& d, const ArmDev& arm, ChainShared& sh, const uint32_t* R,
                               uint32_t* U, uint32_t* so) {
  const int S = arm.S;
  {
    const Box b = sh.box[S];
    const long n = box_words(b);
    for (long t = threadIdx.x; t < n; t += blockDim.x) {
      int wx, y, z;
      box_word(b, t, &wx, &y, &z);
      const long w = ((long)z * d.ny + y) * d.wx + wx;
      U[(long)S * d.nw + w] = R[(long)S * d.nw + w];
    }
  }
  __syncthreads();
  for (int k = S - 1; k >= 0; --k) {
    const Box b = sh.box[k], sb = sh.box[k + 1];
    const SegDev& sg = arm.seg[k];
    const uint32_t* src = U + (long)(k + 1) * d.nw;
    const uint32_t* Rk = R + (long)k * d.nw;
    uint32_t* dst = U + (long)k * d.nw;
    const long n = box_words(b);
    OccBox ob, xb;
    ChainTab tab;
    chain_stage(d, sg, b, sb, sb, src, so, &ob, &xb, &tab);
    for (long t0 = 0; t0 < n; t0 += blockDim.x / kG) {
      const long t = t0 + threadIdx.x / kG;
      int wx = 0, y = 0, z = 0;
      long w = 0;
      uint32_t m = 0;
      if (t < n) {
        box_word(b, t, &wx, &y, &z);
        w = ((long)z * d.ny + y) * d.wx + wx;
        m = Rk[w];
      }
      const uint32_t acc = restricted_word(d, sg, tab, ob, xb, src, sb, wx, y, z, w, m, sh.cnt);
      if (acc && threadIdx.x % kG == 0) dst[w] = acc;
    }
    __syncthreads();
  }
}

// Minimum-index traceback through sets X_0..X_S (X_0 holds the root):
// p_k = min linear index q in X_k with p_{k-1} -> q a valid segment k.
// `coherent` selects plain loads for sets written in this kernel.
template <bool kCoherent>
__device__ bool chain_trace(const Dims& d, const ArmDev& arm, ChainShared& sh, const uint32_t* X,
                            int32_t* pose, uint32_t* so) {
  const int S = arm.S;
  if (threadIdx.x == 0) {
    sh.cur[0] = sh.ref[0][0];
    sh.cur[1] = sh.ref[0][1];
    sh.cur[2] = sh.ref[0][2];
    pose[0] = sh.cur[0];
    pose[1] = sh.cur[1];
    pose[2] = sh.cur[2];
  }
  __syncthreads();
  for (int k = 1; k <= S; ++k) {
    const SegDev& sg = arm.seg[k - 1];
    const uint32_t* Xk = X + (long)k * d.nw;
    const int px = sh.cur[0], py = sh.cur[1], pz = sh.cur[2];
    const long pi = lin(d, px, py, pz);
    if (threadIdx.x == 0) sh.best = ~0ull;
    // the restricted sets lie in the ball boxes: stage the hull of p and box k
    OccBox ob;
    ob.ok = false;
    if (kCoherent) {
      const Box pb{px, px, py, py, pz, pz};
      ob = chain_stage_occ(d, sg, pb, sh.box[k], so);
    }
    __syncthreads();
    const int pwx = px >> 5;
    const long pw = pi >> 5;
    for (int e = threadIdx.x; e < sg.n; e += blockDim.x) {
      const int32_t o = __ldg(sg.off + e);
      const int qx = px + unpack_x(o), qy = py + unpack_y(o), qz = pz + unpack_z(o);
      if (!inside(d, qx, qy, qz)) continue;
      const long qi = lin(d, qx, qy, qz);
      const uint32_t word = kCoherent ? Xk[qi >> 5] : __ldg(Xk + (qi >> 5));
      if (!((word >> (qi & 31)) & 1u)) continue;
      if (!((edge_word_box(d, sg, ob, e, pw, pwx, py, pz) >> (px & 31)) & 1u)) continue;
      atomicMin(&sh.best, (unsigned long long)qi);
    }
    __syncthreads();
    const unsigned long long best = sh.best;
    if (best == ~0ull) return false;
    if (threadIdx.x == 0) {
      const long qi = (long)best;
      sh.cur[0] = (int)(qi % d.nx);
      sh.cur[1] = (int)((qi / d.nx) % d.ny);
      sh.cur[2] = (int)(qi / ((long)d.nx * d.ny));
      pose[3 * k] = sh.cur[0];
      pose[3 * k + 1] = sh.cur[1];
      pose[3 * k + 2] = sh.cur[2];
    }
    __syncthreads();
  }
  return true;
}

// The smooth chain of path p (one block; sh, rad and the dynamic shared
// buffer so of (kChainOccWords + kChainSrcWords) words belong to the caller).
__device__ void smooth_chain_block(const Dims& d, const ArmDev& arm, const ChainArgs& a, int p,
                                   ChainShared& sh, int* rad, uint32_t* so) {
  const int S = arm.S, W = a.W;
  if (threadIdx.x <= IK_MAX_SEG) rad[threadIdx.x] = a.per_joint ? a.rad[threadIdx.x] : a.delta;
  if (threadIdx.x == 0) sh.cnt = a.counters;
  __syncthreads();
  const long pose_sz = 3L * (S + 1);
  int32_t* poses = a.poses + (long)p * W * pose_sz;
  int32_t* relax = a.relax + (long)p * W * 2;
  uint32_t* R = a.scratch + (long)p * 2 * (S + 1) * d.nw;
  uint32_t* U = R + (long)(S + 1) * d.nw;
  const long D2 = (long)(d.nx - 1) * (d.nx - 1) + (long)(d.ny - 1) * (d.ny - 1) +
                  (long)(d.nz - 1) * (d.nz - 1);
  const int cur = a.c_arr ? a.c_arr[p] : a.c;
  if (a.found && !a.found[p]) {
    if (a.mode == 1) return;  // replan slots without work are finished elsewhere
    for (long i = threadIdx.x; i < W * pose_sz; i += blockDim.x) poses[i] = 0;
    for (int i = threadIdx.x; i < 2 * W; i += blockDim.x) relax[i] = -1;
    if (threadIdx.x == 0) a.status[p] = IK_PATH_UNREACHABLE;
    return;
  }
  bool relaxed = false, broken = false;
  int guess = 0;  // search start: the relaxation of the previous waypoint
  const int n_steps = a.mode == 0 ? W - 1 : W - 1 - cur;
  if (threadIdx.x == 0) {
    if (a.mode == 0) {
      relax[2 * (W - 1)] = 0;
      relax[2 * (W - 1) + 1] = 0;
    } else {
      for (int j = 0; j <= cur; ++j) relax[2 * j] = relax[2 * j + 1] = 0;
    }
  }
  for (int s = 0; s < n_steps; ++s) {
    const int j = a.mode == 0 ? W - 2 - s : cur + 1 + s;
    const int rj = a.mode == 0 ? j + 1 : j - 1;
    const uint32_t* V = a.Vw + ((long)p * W + j) * (S + 1) * d.nw;
    int32_t* pose = poses + (long)j * pose_sz;
    const int32_t* refp = poses + (long)rj * pose_sz;
    if (threadIdx.x < (S + 1) * 3) sh.ref[threadIdx.x / 3][threadIdx.x % 3] = refp[threadIdx.x];
    const int eps = a.eps_used[(long)p * W + j];
    if (j < W - 1 && eps != a.relaxed_eps_base) relaxed = true;
    __syncthreads();
    if (threadIdx.x == 0) relax[2 * j + 1] = eps;
    const bool vok = inside(d, sh.ref[0][0], sh.ref[0][1], sh.ref[0][2]) &&
                     test_bit(V, lin(d, sh.ref[0][0], sh.ref[0][1], sh.ref[0][2]));
    int m_star = -1;
    // R holds the forward restriction of the last feasibility test (boxes in
    // sh.box) when r_for >= 0; dirty: R / U hold words that must be cleared
    int r_for = -1;
    bool dirty = false;
    const int32_t* vb = a.vbox ? a.vbox + ((long)p * W + j) * (S + 1) * 6 : nullptr;
    // every filtered joint's ball covers the grid ((rad + m)^2 >= D2)
    auto covers = [&](int m) {
      for (int k = 1; k <= S; ++k)
        if (rad[k] >= 0 && (long)(rad[k] + m) * (rad[k] + m) < D2) return false;
      return true;
    };
    // Is there a chain inside the balls of radius rad + m?  Once the balls
    // cover the grid there is, because V is non-empty.
    auto feasible = [&](int m) {
      if (covers(m)) return true;
      if (dirty) chain_clear(d, sh, S, R, U);
      chain_boxes(d, sh, S, m, rad, vb);
      dirty = true;
      if (sh.empty) {
        r_for = -1;
        return false;
      }
      const bool ok = chain_forward(d, arm, sh, V, R, so);
      r_for = ok ? m : -1;
      return ok;
    };
    if (vok) {
      // Smallest m with a chain inside the balls of radius delta + m (at most
      // max_relax when that is bounded).  Feasibility only grows with m, so
      // any search that brackets the smallest feasible m finds the same m as
      // trying m = 0, 1, 2, ... in turn.  The search starts next to the
      // previous waypoint's m, which consecutive waypoints usually share:
      // gallop down or up from there, then bisect.
      const int cap = a.max_relax >= 0 ? a.max_relax : 0x3fffffff;
      int lo = -1, hi = -1;
      const int g = min(guess, cap);
      if (g > 0) {
        if (feasible(g - 1)) hi = g - 1;
        else lo = g - 1;
      }
      if (hi < 0) {
        for (int step = 1;; step *= 2) {
          if (lo >= cap) break;
          const int m = (int)min((long)lo + step, (long)cap);
          if (feasible(m)) {
            hi = m;
            break;
          }
          lo = m;
        }
      } else {
        for (int step = 1; hi > 0; step *= 2) {
          const int m = max(hi - step, 0);
          if (!feasible(m)) {
            lo = m;
            break;
          }
          hi = m;
        }
      }
      if (hi >= 0) {
        while (hi - lo > 1) {
          const int mid = lo + (hi - lo) / 2;
          if (feasible(mid)) hi = mid;
          else lo = mid;
        }
      }
      m_star = hi;
    }
    bool done = false;
    if (m_star >= 0) {
      guess = m_star;
      if (covers(m_star)) {
        if (dirty) chain_clear(d, sh, S, R, U);
        dirty = false;
        done = chain_trace<false>(d, arm, sh, V, pose, so);
      } else {
        bool ok = true;
        if (r_for != m_star) ok = feasible(m_star);  // the last test was another m
        if (ok) {
          chain_backward(d, arm, sh, R, U, so);
          done = chain_trace<true>(d, arm, sh, U, pose, so);
        }
      }
    }
    if (dirty) chain_clear(d, sh, S, R, U);
    if (done) {
      if (m_star > 0) relaxed = true;
      if (threadIdx.x == 0) relax[2 * j] = m_star;
    } else {
      broken = true;
      for (int i = threadIdx.x; i < pose_sz; i += blockDim.x) pose[i] = refp[i];
      if (threadIdx.x == 0) relax[2 * j] = -1;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0)
    a.status[p] = broken ? IK_PATH_BROKEN : (relaxed ? IK_PATH_RELAXED : IK_PATH_OK);
}

__global__ void __launch_bounds__(kChainThreads, 1) k_smooth_chain(Dims d, ArmDev arm, ChainArgs a) {
  __shared__ ChainShared sh;
  __shared__ int rad[IK_MAX_SEG + 1];  // filter radius of each joint (-1: none)
  extern __shared__ uint32_t so[];
  smooth_chain_block(d, arm, a, blockIdx.x, sh, rad, so);
}

// ------------------------------------------------- folded last segment

// One block per (path, waypoint): the pose's joints 0 .. F come from the
// follower chain (tposes); joint F + 1 = S is the end of the last segment
// from the follower f: among the admissible, obstacle-free offsets of
// segment S that end inside the grid, the end q nearest to the fold point
// A / den (|den q - A|^2), then the smallest linear index.  Without one the
// end stays at f, the waypoint records -1 and the path is broken.
__global__ void k_fold_last(Dims d, SegDev sg, int S, int W, const int32_t* __restrict__ tposes,
                            const int32_t* __restrict__ fold_at, int32_t* __restrict__ poses,
                            int32_t* __restrict__ relax, int32_t* __restrict__ status) {
  const int j = blockIdx.x, p = blockIdx.y, F = S - 1;
  const int32_t* tp = tposes + ((long)p * W + j) * 3 * (F + 1);
  int32_t* out = poses + ((long)p * W + j) * 3 * (S + 1);
  const int32_t* fa = fold_at + ((long)p * W + j) * 4;
  __shared__ unsigned long long best_key, best_idx;
  if (threadIdx.x == 0) {
    best_key = ~0ull;
    best_idx = ~0ull;
  }
  for (int i = threadIdx.x; i < 3 * (F + 1); i += blockDim.x) out[i] = tp[i];
  __syncthreads();
  const int fx = tp[3 * F], fy = tp[3 * F + 1], fz = tp[3 * F + 2];
  const long fi = lin(d, fx, fy, fz);
  const long den = fa[3];
  // pass 1: the smallest distance key; pass 2: the smallest index at that key
  for (int pass = 0; pass < 2; ++pass) {
    for (int e = threadIdx.x; e < sg.n; e += blockDim.x) {
      const int32_t o = __ldg(sg.off + e);
      const int qx = fx + unpack_x(o), qy = fy + unpack_y(o), qz = fz + unpack_z(o);
      if (!inside(d, qx, qy, qz)) continue;
      const long ex = den * qx - fa[0], ey = den * qy - fa[1], ez = den * qz - fa[2];
      const unsigned long long key = (unsigned long long)(ex * ex + ey * ey + ez * ez);
      if (pass == 0 ? key >= best_key : key != best_key) continue;
      if (!edge_bit(d, sg, e, fi)) continue;
      if (pass == 0)
        atomicMin(&best_key, key);
      else
        atomicMin(&best_idx, (unsigned long long)lin(d, qx, qy, qz));
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (best_idx == ~0ull) {
      out[3 * S] = fx;
      out[3 * S + 1] = fy;
      out[3 * S + 2] = fz;
      relax[((long)p * W + j) * 2] = -1;
      status[p] = IK_PATH_BROKEN;  // every writer stores the same value
    } else {
      const long qi = (long)best_idx;
      out[3 * S] = (int)(qi % d.nx);
      out[3 * S + 1] = (int)((qi / d.nx) % d.ny);
      out[3 * S + 2] = (int)(qi / ((long)d.nx * d.ny));
    }
  }
}

cudaError_t launch_fold_last(const Dims& d, const SegDev& sg, int S, int P, int W, const int32_t* tposes,
                             const int32_t* fold_at, int32_t* poses, int32_t* relax, int32_t* status,
                             cudaStream_t st) {
  if (P <= 0 || W <= 0) return cudaSuccess;
  k_fold_last<<<dim3(W, P), 256, 0, st>>>(d, sg, S, W, tposes, fold_at, poses, relax, status);
  return cudaGetLastError();
}

cudaError_t set_kernel_attributes() {
  // opt in to large dynamic shared memory for the tiled kernels (per device;
  // called when a grid is created, never during stream capture)
  const int bytes = 200 * 1024;
  cudaError_t e = cudaFuncSetAttribute((const void*)k_edge_masks_tile,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute((const void*)k_edge_masks_tma, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kTileOccSmemMax);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute((const void*)k_propagate_tile_pair<true, false, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, kTileOccSmemMax);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute((const void*)k_propagate_tile_pair<false, false, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, kTileOccSmemMax);
  if (e == cudaSuccess) e = set_rows_attributes<1>();
  {
    const void* fns[] = {(const void*)k_edge_masks_rows<1, false>, (const void*)k_edge_masks_rows<1, true>,
                         (const void*)k_edge_masks_rows<2, false>, (const void*)k_edge_masks_rows<2, true>,
                         (const void*)k_edge_masks_rows<4, false>, (const void*)k_edge_masks_rows<4, true>,
                         (const void*)k_edge_masks_rows<8, false>, (const void*)k_edge_masks_rows<8, true>};
    for (const void* f : fns)
      if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, kTileOccSmemMax);
  }
  if (e == cudaSuccess) e = set_rows_attributes<2>();
  if (e == cudaSuccess) e = set_rows_attributes<4>();
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute((const void*)k_propagate_tile_pair<true, false>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, kTileOccSmemMax);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute((const void*)k_propagate_tile_pair<false, false>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, kTileOccSmemMax);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute((const void*)k_propagate_tile_pair<true, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, kTileOccSmemMax);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute((const void*)k_propagate_tile_pair<false, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, kTileOccSmemMax);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute((const void*)k_propagate_tile<true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute((const void*)k_propagate_tile<false>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute((const void*)k_propagate_tile_list<true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute((const void*)k_propagate_tile_list<false>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute((const void*)k_propagate_tile_occ_list<true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, kTileOccSmemMax);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute((const void*)k_propagate_tile_occ_list<false>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, kTileOccSmemMax);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute((const void*)k_propagate_tile_occ<true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, kTileOccSmemMax);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute((const void*)k_propagate_tile_occ<false>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, kTileOccSmemMax);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute((const void*)k_smooth_chain, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)((kChainOccWords + kChainSrcWords) * sizeof(uint32_t)));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute((const void*)k_propagate_tile2<true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute((const void*)k_propagate_tile2<false>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  return e;
}

cudaError_t launch_smooth_chain(const Dims& d, const ArmDev& arm, const ChainArgs& a,
                                cudaStream_t st) {
  if (a.P <= 0) return cudaSuccess;
  k_smooth_chain<<<a.P, kChainThreads, (kChainOccWords + kChainSrcWords) * sizeof(uint32_t), st>>>(d, arm,
                                                                                                   a);
  return cudaGetLastError();
}

// The persistent uneven-batch kernel uses the block bodies above.
#include "ik_batch_kernel.cuh"

}  // namespace ikb
