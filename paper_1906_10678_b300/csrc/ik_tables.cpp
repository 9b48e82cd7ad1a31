// Host-side construction of the per-segment tables: the shell of admissible
// offsets and each offset's closed supercover.
//
// The shell replaces the paper's quiver (section "Discretization of the
// segment articulations": unit directions times the segment length) by every
// integer offset whose length is within tol of the segment length; the
// supercover replaces the n equispaced collision sample points of section
// "Testing for collisions" by every voxel whose closed cube meets the
// segment, so that no obstacle voxel can slip between sample points.

#include <algorithm>
#include <cstdlib>
#include <array>
#include <cmath>

#include "ik_internal.h"

namespace ikb {

void shell_bounds(int len, double tol, int* lo2, int* hi2) {
  double a = (double)len - tol;
  double b = (double)len + tol;
  double lo = (a > 0.0) ? std::ceil(a * a) : 0.0;
  *lo2 = std::max(1, (int)lo);
  *hi2 = (int)std::floor(b * b);
}

static int isqrt_floor(long v) {  // largest r with r*r <= v, v >= 0
  long r = (long)std::sqrt((double)v);
  while (r * r > v) --r;
  while ((r + 1) * (r + 1) <= v) ++r;
  return (int)r;
}

static int isqrt_ceil(long v) {  // smallest r >= 0 with r*r >= v
  if (v <= 0) return 0;
  int r = isqrt_floor(v);
  return (long)r * r == v ? r : r + 1;
}

// Closed supercover of the segment 0 -> d by walking its boundary
// crossings.  Along axis i the segment t*d crosses the voxel faces
// x_i = s_i (k + 1/2), k = 0 .. |d_i| - 1, at t = (2k + 1) / (2 |d_i|).
// Crossings are visited in increasing t (exact integer comparison).  At a
// crossing time shared by the axes in A, the segment point lies on the faces
// of every voxel cur + sum_{i in B} s_i e_i for B a subset of A, so all of
// them are touched; then the walk steps to cur + sum_{i in A} s_i e_i.  The
// voxels go to out (capacity cap, no allocation), sorted by (z, y, x)
// without repeats; returns their number, or -1 when they do not fit.
int supercover_walk(int dx, int dy, int dz, int32_t* out, int cap) {
  const int d[3] = {dx, dy, dz};
  int n[3], s[3], k[3] = {0, 0, 0}, cur[3] = {0, 0, 0};
  for (int i = 0; i < 3; ++i) {
    n[i] = d[i] < 0 ? -d[i] : d[i];
    s[i] = d[i] < 0 ? -1 : 1;
  }
  int cnt = 0;
  auto push = [&](int x, int y, int z) {
    if (cnt < cap) out[cnt] = pack3(x, y, z);
    ++cnt;
  };
  push(0, 0, 0);
  for (;;) {
    // earliest pending crossing: compare (2k_i+1)/(2n_i) by cross-multiplying
    int best = -1;
    for (int i = 0; i < 3; ++i) {
      if (k[i] >= n[i]) continue;
      if (best < 0 || (long)(2 * k[i] + 1) * n[best] < (long)(2 * k[best] + 1) * n[i]) best = i;
    }
    if (best < 0) break;
    int A[3], na = 0;
    for (int i = 0; i < 3; ++i)
      if (k[i] < n[i] && (long)(2 * k[i] + 1) * n[best] == (long)(2 * k[best] + 1) * n[i]) A[na++] = i;
    for (int mask = 1; mask < (1 << na); ++mask) {
      int v[3] = {cur[0], cur[1], cur[2]};
      for (int b = 0; b < na; ++b)
        if (mask & (1 << b)) v[A[b]] += s[A[b]];
      push(v[0], v[1], v[2]);
    }
    for (int b = 0; b < na; ++b) {
      cur[A[b]] += s[A[b]];
      ++k[A[b]];
    }
  }
  if (cnt > cap) return -1;
  // (z, y, x) order (the key keeps it: |x|, |y| < 512), then drop repeats;
  // insertion sort, the lists are short
  auto key = [](int32_t v) { return ((long)unpack_z(v) << 20) + ((long)unpack_y(v) << 10) + unpack_x(v); };
  for (int i = 1; i < cnt; ++i) {
    const int32_t v = out[i];
    int j = i - 1;
    while (j >= 0 && key(out[j]) > key(v)) {
      out[j + 1] = out[j];
      --j;
    }
    out[j + 1] = v;
  }
  int u = 0;
  for (int i = 0; i < cnt; ++i)
    if (u == 0 || out[u - 1] != out[i]) out[u++] = out[i];
  return u;
}

void supercover_traverse(int dx, int dy, int dz, std::vector<int32_t>* out) {
  // at most one voxel per crossing subset: 1 + 7 (|dx| + |dy| + |dz|)
  const int cap = 8 + 7 * (std::abs(dx) + std::abs(dy) + std::abs(dz));
  out->resize(cap);
  const int n = supercover_walk(dx, dy, dz, out->data(), cap);
  out->resize(n < 0 ? 0 : n);
}

static bool cone_keeps(const ConeSpec& c, long x, long y, long z) {
  const long proj = x * c.ax + y * c.ay + z * c.az;
  if (proj <= 0) return false;
  const long n2 = x * x + y * y + z * z;
  const long a2 = (long)c.ax * c.ax + (long)c.ay * c.ay + (long)c.az * c.az;
  return (long)c.den * proj * proj >= (long)c.num * n2 * a2;
}

void build_shell(int lo2, int hi2, ShellHost* sh, const ConeSpec* cone) {
  struct Off {
    int x, y, z, n2;
  };
  std::vector<Off> offs;
  const int R = isqrt_floor(hi2);
  for (int z = -R; z <= R; ++z) {
    for (int y = -R; y <= R; ++y) {
      long yz = (long)y * y + (long)z * z;
      if (yz > hi2) continue;
      int xmin = isqrt_ceil(std::max(0L, (long)lo2 - yz));
      int xmax = isqrt_floor(hi2 - yz);
      if (xmin > xmax) continue;
      for (int x = -xmax; x <= xmax; ++x) {
        int ax = x < 0 ? -x : x;
        if (ax < xmin) continue;
        if (cone && !cone_keeps(*cone, x, y, z)) continue;
        offs.push_back({x, y, z, (int)(x * x + yz)});
      }
    }
  }
  std::sort(offs.begin(), offs.end(), [](const Off& a, const Off& b) {
    if (a.n2 != b.n2) return a.n2 < b.n2;
    if (a.z != b.z) return a.z < b.z;
    if (a.y != b.y) return a.y < b.y;
    return a.x < b.x;
  });
  sh->lo2 = lo2;
  sh->hi2 = hi2;
  sh->off.clear();
  for (const Off& o : offs) sh->off.push_back(pack3(o.x, o.y, o.z));
  // device order (z, y, x) with a row table over (dz, dy)
  std::vector<Off> dev = offs;
  std::sort(dev.begin(), dev.end(), [](const Off& a, const Off& b) {
    if (a.z != b.z) return a.z < b.z;
    if (a.y != b.y) return a.y < b.y;
    return a.x < b.x;
  });
  sh->R = R;
  const int side = 2 * R + 1;
  sh->rows.assign((size_t)side * side + 1, 0);
  std::vector<int32_t> count((size_t)side * side, 0);
  for (const Off& o : dev) ++count[(size_t)(o.z + R) * side + (o.y + R)];
  for (size_t r = 0; r < count.size(); ++r) sh->rows[r + 1] = sh->rows[r] + count[r];
  sh->dev_off.clear();
  sh->sc.clear();
  sh->sc_start.assign(1, 0);
  sh->max_sc = 0;
  std::vector<int32_t> sc;
  for (const Off& o : dev) {
    sh->dev_off.push_back(pack3(o.x, o.y, o.z));
    supercover_traverse(o.x, o.y, o.z, &sc);
    sh->sc.insert(sh->sc.end(), sc.begin(), sc.end());
    sh->sc_start.push_back((int32_t)sh->sc.size());
    sh->max_sc = std::max(sh->max_sc, (int)sc.size());
  }
}

TileCfg make_tile_cfg(const Dims& d) {
  TileCfg tc;
  tc.TY = 32 / d.wx;
  tc.lanes = tc.TY * d.wx;
  tc.TZ = 8;
  tc.tiles_y = (d.ny + tc.TY - 1) / tc.TY;
  tc.tiles_z = (d.nz + tc.TZ - 1) / tc.TZ;
  // Pitch of a staged row (words): the narrowest with at most 2-way bank
  // conflicts among a warp's 32 row-word addresses (at least the row width
  // plus the two halo words, at most 31 so that a row fits one warp).  A
  // narrow halo lets more blocks share an SM, which measured faster than a
  // conflict-free pitch (twice as wide on the 128^3 grid: 90 vs 105 ms per
  // step).
  auto degree = [&](int P) {
    int hits[32] = {0}, conf = 0;
    for (int l = 0; l < tc.lanes; ++l) conf = std::max(conf, ++hits[((l / d.wx) * P + (l % d.wx)) & 31]);
    return conf;
  };
  int best = -1;
  for (int P = d.wx + 2; P <= 31 && best < 0; ++P)
    if (degree(P) <= 2) best = P;
  // rows of 30 words or more do not fit: the pitch then exceeds 31 and the
  // tiled kernels stand aside (tile_smem_bytes and its kin return 0)
  if (best < 0) best = d.wx + 2;
  tc.P = best;
  return tc;
}

size_t tile_smem_bytes(const TileCfg& tc, int R) {
  if (R > 31) return 0;     // the x halo would exceed one word
  if (tc.P > 31) return 0;  // a staged row must fit in one warp's lanes
  const size_t bytes = (size_t)(tc.TZ + 2 * R) * (tc.TY + 2 * R) * tc.P * 4;
  return bytes <= 200 * 1024 ? bytes : 0;
}

size_t tile_occ_smem_bytes(const TileCfg& tc, int R) {
  if (R > 31 || tc.P > 31) return 0;
  const size_t bytes = 2 * (size_t)(tc.TZ + 2 * R) * (tc.TY + 2 * R) * tc.P * 4;
  return bytes <= (size_t)kTileOccSmemMax ? bytes : 0;
}

}  // namespace ikb
