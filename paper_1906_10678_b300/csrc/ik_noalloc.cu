// Forward reachable sets without any allocation.
//
// Some callers cannot allocate GPU memory at the point where they need an
// answer: code running under a caching or arena allocator that owns the whole
// device, real-time loops where cudaMalloc/cudaFree would synchronise the
// device or stall unpredictably, and hosts that forbid allocation after
// start-up.  ik_forward_sets_noalloc serves them: the caller passes the
// occupancy and the output sets (device memory it already owns); the
// library's scratch -- the arm's shell offsets and supercover lists -- lives
// in one file-scope __device__ array of fixed size, and neither this file's
// host code nor its kernel allocates device or host memory.  Edge masks are
// not stored: each segment test walks its supercover against the occupancy.

#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <cmath>
#include <mutex>

#include "ik_internal.h"

namespace {

// Scratch limits (words): shell offsets of all segments, their supercover
// start indices, and the supercover voxels.
constexpr int kNaMaxOff = 32768;
constexpr int kNaMaxSc = 1 << 20;
constexpr int kNaWords = kNaMaxOff + (kNaMaxOff + IK_MAX_SEG) + kNaMaxSc;  // 4.25 MiB
constexpr int kNaMaxDevices = 64;

// The scratch array.  Every call on a device shares it and it keeps the last
// call's contents; calls whose work overlaps on the GPU race on it.
static __device__ __align__(256) int32_t g_na_scratch[kNaWords];

// Device addresses of g_na_scratch, one per device, fetched on first use.
int32_t* g_na_addr[kNaMaxDevices] = {nullptr};

// Host staging of the tables (fixed size; no heap).  g_na_mutex (which
// allocates nothing) serialises host threads from the first use of g_na_addr
// through the last copy out of these tables; a pageable-source
// cudaMemcpyAsync has consumed its source when it returns.
std::mutex g_na_mutex;
int32_t h_na_off[kNaMaxOff];
int32_t h_na_start[kNaMaxOff + IK_MAX_SEG];
int32_t h_na_sc[kNaMaxSc];

struct NaSeg {
  int off0, n;  // offsets [off0, off0 + n) of the scratch offset table
  int lo2, hi2;
};

struct NaArm {
  NaSeg seg[IK_MAX_SEG];
  int S;
};

// Fill the host staging tables for the arm; IK_ERR_UNSUPPORTED when they
// exceed the scratch limits.
int na_tables(const ik_arm* arm, NaArm* na, int* n_off, int* n_sc) {
  int o = 0, c = 0;
  na->S = arm->n_seg;
  for (int k = 0; k < arm->n_seg; ++k) {
    int lo2, hi2;
    ikb::shell_bounds(arm->len[k], (double)arm->tol, &lo2, &hi2);
    if (hi2 < lo2) return IK_ERR_ARG;
    na->seg[k].off0 = o;
    na->seg[k].lo2 = lo2;
    na->seg[k].hi2 = hi2;
    int R = 0;
    while ((R + 1) * (R + 1) <= hi2) ++R;
    for (int z = -R; z <= R; ++z)
      for (int y = -R; y <= R; ++y)
        for (int x = -R; x <= R; ++x) {
          const int n2 = x * x + y * y + z * z;
          if (n2 < lo2 || n2 > hi2) continue;
          if (o >= kNaMaxOff) return IK_ERR_UNSUPPORTED;
          h_na_off[o] = ikb::pack3(x, y, z);
          h_na_start[o] = c;
          const int m = ikb::supercover_walk(x, y, z, h_na_sc + c, kNaMaxSc - c);
          if (m < 0) return IK_ERR_UNSUPPORTED;
          c += m;
          ++o;
        }
    na->seg[k].n = o - na->seg[k].off0;
  }
  h_na_start[o] = c;
  *n_off = o;
  *n_sc = c;
  return IK_OK;
}

__device__ __forceinline__ uint32_t na_shifted(const uint32_t* __restrict__ s, const ikb::Dims& d, int wx,
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

// F_0 = {root} if free.
__global__ void k_na_seed(ikb::Dims d, const uint32_t* __restrict__ occ, int rx, int ry, int rz,
                          uint32_t* __restrict__ F0) {
  const long w = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (w >= d.nw) return;
  const long i = ((long)rz * d.ny + ry) * d.nx + rx;
  const uint32_t v = ((i >> 5) == w) ? (1u << (i & 31)) : 0u;
  F0[w] = v & ~__ldg(occ + w);
}

// F_k[p] = OR_e F_{k-1}[p + e] & (segment p -> p + e free), the segment test
// made on the fly from the supercover list of e (tables in the scratch).
__global__ void __launch_bounds__(256) k_na_forward(ikb::Dims d, const uint32_t* __restrict__ occ,
                                                    const int32_t* __restrict__ tab, NaSeg seg,
                                                    const uint32_t* __restrict__ X,
                                                    uint32_t* __restrict__ out) {
  const long w = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (w >= d.nw) return;
  const int32_t* off = tab;
  const int32_t* start = tab + kNaMaxOff;
  const int32_t* sc = tab + kNaMaxOff + kNaMaxOff + IK_MAX_SEG;
  const int wx = (int)(w % d.wx), y = (int)((w / d.wx) % d.ny), z = (int)(w / ((long)d.wx * d.ny));
  const uint32_t m = ~__ldg(occ + w);
  uint32_t acc = 0;
  for (int e = seg.off0; e < seg.off0 + seg.n && (acc & m) != m; ++e) {
    const int32_t o = __ldg(off + e);
    const uint32_t x = na_shifted(X, d, wx, y, z, ikb::unpack_x(o), ikb::unpack_y(o), ikb::unpack_z(o));
    if (!(x & m & ~acc)) continue;
    uint32_t blocked = 0;
    const int s1 = __ldg(start + e + 1);
    for (int i = __ldg(start + e); i < s1 && blocked != 0xffffffffu; ++i) {
      const int32_t v = __ldg(sc + i);
      blocked |= na_shifted(occ, d, wx, y, z, ikb::unpack_x(v), ikb::unpack_y(v), ikb::unpack_z(v));
    }
    acc |= x & ~blocked;
  }
  out[w] = acc & m;
}

int na_fail(cudaError_t e) {
  cudaGetLastError();  // clear a non-sticky error so later calls start clean
  return e == cudaErrorMemoryAllocation ? IK_ERR_OOM : IK_ERR_CUDA;
}

}  // namespace

extern "C" {

int ik_forward_sets_noalloc(const uint32_t* occ_words, int nx, int ny, int nz, const ik_arm* arm,
                            const int32_t root[3], uint32_t* fsets_out, void* cuda_stream) {
  if (!occ_words || !fsets_out || !arm || !arm->len || !root) return IK_ERR_ARG;
  if (nx < 32 || nx > 1024 || nx % 32 != 0 || ny < 1 || ny > 1024 || nz < 1 || nz > 1024)
    return IK_ERR_ARG;
  if (arm->n_seg < 1 || arm->n_seg > IK_MAX_SEG || !(arm->tol >= 0.0f && arm->tol < 1.0f))
    return IK_ERR_ARG;
  for (int k = 0; k < arm->n_seg; ++k)
    if (arm->len[k] < 1 || arm->len[k] > IK_MAX_LEN) return IK_ERR_ARG;
  if (root[0] < 0 || root[1] < 0 || root[2] < 0 || root[0] >= nx || root[1] >= ny || root[2] >= nz)
    return IK_ERR_ARG;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return na_fail(e);
  if (dev < 0 || dev >= kNaMaxDevices) return IK_ERR_UNSUPPORTED;
  std::unique_lock<std::mutex> lock(g_na_mutex);
  if (!g_na_addr[dev]) {
    // once per device, with that device current: the host-side symbol is a
    // stand-in, the kernels need the device address
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_na_scratch);
    if (e != cudaSuccess) return na_fail(e);
    g_na_addr[dev] = (int32_t*)p;
  }
  int32_t* scratch = g_na_addr[dev];
  NaArm na;
  int n_off = 0, n_sc = 0;
  int rc = na_tables(arm, &na, &n_off, &n_sc);
  if (rc) return rc;
  // the scratch keeps the previous call's tables: overwrite every part used
  e = cudaMemcpyAsync(scratch, h_na_off, (size_t)n_off * 4, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(scratch + kNaMaxOff, h_na_start, (size_t)(n_off + 1) * 4,
                        cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(scratch + 2 * kNaMaxOff + IK_MAX_SEG, h_na_sc, (size_t)n_sc * 4,
                        cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return na_fail(e);
  lock.unlock();  // the host tables are consumed; the kernels read the device scratch
  ikb::Dims d;
  d.nx = nx;
  d.ny = ny;
  d.nz = nz;
  d.wx = nx / 32;
  d.nw = (long)d.wx * ny * nz;
  const int grid = (int)((d.nw + 255) / 256);
  k_na_seed<<<grid, 256, 0, st>>>(d, occ_words, root[0], root[1], root[2], fsets_out);
  for (int k = 1; k <= na.S; ++k)
    k_na_forward<<<grid, 256, 0, st>>>(d, occ_words, scratch, na.seg[k - 1],
                                        fsets_out + (long)(k - 1) * d.nw, fsets_out + (long)k * d.nw);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return na_fail(e);
  return IK_OK;
}

}  // extern "C"
