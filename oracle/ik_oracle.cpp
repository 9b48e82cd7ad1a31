// ORACLE — test infrastructure, not product code.
//
// A plain, slow, obviously-correct CPU restatement of the gap map-seeking
// (gMS) inverse-kinematics search and its path planner (Arathorn,
// arXiv 1906.10678), in the exact lattice form used throughout this project:
//
//   * joints live on voxel centres of an Nx x Ny x Nz grid (index
//     iota = (z*Ny + y)*Nx + x), obstacles are voxels marked 1;
//   * a segment of nominal length L may take any integer offset d with
//     lo2 <= |d|^2 <= hi2, lo2 = max(1, ceil((L-tol)^2)), hi2 = floor((L+tol)^2)
//     (the "shell"; it stands in for the quiver of directions times the
//     segment length, section "Discretization of the segment articulations",
//     and for the epsilon on the gap vector's length, section "The gap in gMS");
//   * a segment p->q is obstacle-free when every voxel of its closed
//     supercover (voxels whose closed unit cube meets the closed segment) is
//     free (stands in for the n sample points of section "Testing for
//     collisions");
//   * Step 1 / Step 2A of "The procedure for IK solution" become forward
//     reachable sets F_k grown from the root, the backward (cone) mapping from
//     the target becomes backward sets B_k, the gap test becomes V_k = F_k & B_k,
//     and Step 3's choice of one surviving chain becomes a minimum-linear-index
//     traceback.
//
// Every set is a byte per voxel (no bit packing), every segment test walks
// its supercover voxel by voxel, and every step follows the definitions in
// the order they are stated.  Only tests/, the smoke check and the benchmark's
// CPU-baseline leg load this library; the product path never does.
//
// Parity status: supercover, shells, F/B/V sets and the reach traceback are
// pinned by brute-force chain enumeration, closed forms and worked examples
// (tests/test_oracle_pins.py).  The path planner and replanner follow
// rules that the paper states only in words (sections "Smooth sequence
// computation", "Filtering for smoothness", "Dynamic Obstacles"); they are
// pinned by brute force over restricted balls on tiny grids (the replanner
// on every branch, its reach re-solve against a lexicographic minimum over
// all enumerated chains) and by invariants, not by any number printed in
// the paper.  The word-pair count is pinned by a numpy shift-and-pack count.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

namespace {

struct Grid {
  int nx, ny, nz;
  long nvox() const { return (long)nx * ny * nz; }
  bool inside(int x, int y, int z) const {
    return x >= 0 && y >= 0 && z >= 0 && x < nx && y < ny && z < nz;
  }
  long index(int x, int y, int z) const { return ((long)z * ny + y) * nx + x; }
};

struct V3 {
  int x, y, z;
};

static inline long sq(long v) { return v * v; }
static inline long dist2(const V3& a, const V3& b) {
  return sq(a.x - b.x) + sq(a.y - b.y) + sq(a.z - b.z);
}

// ---------------------------------------------------------------------------
// Shell of admissible segment offsets for one segment length.
// ---------------------------------------------------------------------------

// Integer bounds of the shell: lo2 = ceil((L - tol)^2) (at least 1, so the
// zero offset never counts as a segment) and hi2 = floor((L + tol)^2),
// evaluated in IEEE double precision.
static void shell_bounds(int L, double tol, int* lo2, int* hi2) {
  double a = (double)L - tol;
  double b = (double)L + tol;
  double lo = (a > 0.0) ? std::ceil(a * a) : 0.0;
  double hi = std::floor(b * b);
  *lo2 = std::max(1, (int)lo);
  *hi2 = (int)hi;
}

// All d with lo2 <= |d|^2 <= hi2, ordered by (|d|^2, z, y, x).
static std::vector<V3> shell(int lo2, int hi2) {
  std::vector<V3> out;
  int R = 0;
  while ((long)(R + 1) * (R + 1) <= hi2) ++R;
  for (int z = -R; z <= R; ++z)
    for (int y = -R; y <= R; ++y)
      for (int x = -R; x <= R; ++x) {
        long n2 = (long)x * x + (long)y * y + (long)z * z;
        if (n2 >= lo2 && n2 <= hi2) out.push_back({x, y, z});
      }
  std::stable_sort(out.begin(), out.end(), [](const V3& a, const V3& b) {
    long na = (long)a.x * a.x + (long)a.y * a.y + (long)a.z * a.z;
    long nb = (long)b.x * b.x + (long)b.y * b.y + (long)b.z * b.z;
    if (na != nb) return na < nb;
    if (a.z != b.z) return a.z < b.z;
    if (a.y != b.y) return a.y < b.y;
    return a.x < b.x;
  });
  return out;
}

// ---------------------------------------------------------------------------
// Closed supercover by an exact rational slab test.
// ---------------------------------------------------------------------------

// Fraction num/den with den > 0.
struct Frac {
  long n, d;
};
static inline bool frac_lt(const Frac& a, const Frac& b) { return a.n * b.d < b.n * a.d; }

// Does the closed unit cube centred on voxel c meet the closed segment a->b?
// The segment is a + t (b - a), t in [0, 1].  Along axis i the point stays in
// the cube's slab |a_i + t d_i - c_i| <= 1/2, i.e. 2u - 1 <= 2 t d_i <= 2u + 1
// with u = c_i - a_i.  The cube meets the segment iff the intersection of the
// per-axis t-intervals with [0, 1] is non-empty.
static bool cube_meets_segment(const V3& a, const V3& b, const V3& c) {
  Frac lo{0, 1}, hi{1, 1};
  const int av[3] = {a.x, a.y, a.z};
  const int bv[3] = {b.x, b.y, b.z};
  const int cv[3] = {c.x, c.y, c.z};
  for (int i = 0; i < 3; ++i) {
    long d = (long)bv[i] - av[i];
    long u = (long)cv[i] - av[i];
    if (d == 0) {
      if (u != 0) return false;  // |u| <= 1/2 with integer u
      continue;
    }
    Frac l, h;
    if (d > 0) {
      l = {2 * u - 1, 2 * d};
      h = {2 * u + 1, 2 * d};
    } else {
      l = {-(2 * u + 1), -2 * d};
      h = {-(2 * u - 1), -2 * d};
    }
    if (frac_lt(lo, l)) lo = l;
    if (frac_lt(h, hi)) hi = h;
  }
  return !frac_lt(hi, lo);
}

// Supercover of the segment a->b: every voxel of the bounding box of {a, b}
// whose cube meets the segment, in (z, y, x) order.  (A voxel outside the
// bounding box is at least one unit away along some axis, so its cube
// cannot meet the segment.)
static std::vector<V3> supercover(const V3& a, const V3& b) {
  std::vector<V3> out;
  for (int z = std::min(a.z, b.z); z <= std::max(a.z, b.z); ++z)
    for (int y = std::min(a.y, b.y); y <= std::max(a.y, b.y); ++y)
      for (int x = std::min(a.x, b.x); x <= std::max(a.x, b.x); ++x) {
        V3 c{x, y, z};
        if (cube_meets_segment(a, b, c)) out.push_back(c);
      }
  return out;
}

// ---------------------------------------------------------------------------
// Arm: one shell per segment, each offset with its supercover from the origin.
// SC(p, p+d) = p + SC(0, d) because the slab test depends only on
// differences; the tests pin that identity directly.
// ---------------------------------------------------------------------------

struct Segment {
  int lo2, hi2;
  std::vector<V3> offs;               // the shell
  std::vector<std::vector<V3>> sc;    // sc[i] = SC(0, offs[i])
};

static Segment make_segment(int lo2, int hi2) {
  Segment s;
  s.lo2 = lo2;
  s.hi2 = hi2;
  s.offs = shell(lo2, hi2);
  s.sc.reserve(s.offs.size());
  V3 o{0, 0, 0};
  for (const V3& d : s.offs) s.sc.push_back(supercover(o, d));
  return s;
}

struct Problem {
  Grid g;
  const uint8_t* occ;  // 1 = occupied
  std::vector<Segment> seg;  // seg[k-1] is segment k
  int S() const { return (int)seg.size(); }
};

// Segment k placed at p with offset number i: every supercover voxel free?
// (Both endpoints are assumed inside the grid, so the supercover is too.)
static bool edge_free(const Problem& P, const V3& p, const std::vector<V3>& sc) {
  for (const V3& v : sc) {
    if (P.occ[P.g.index(p.x + v.x, p.y + v.y, p.z + v.z)]) return false;
  }
  return true;
}

// d is one of the segment's admissible offsets (its shell, or the part of it
// that a direction limit keeps).
static bool is_offset_in_shell(const Segment& s, const V3& d) {
  for (const V3& o : s.offs)
    if (o.x == d.x && o.y == d.y && o.z == d.z) return true;
  return false;
}

static inline V3 at(const Grid& g, long i) {
  V3 v;
  v.x = (int)(i % g.nx);
  v.y = (int)((i / g.nx) % g.ny);
  v.z = (int)(i / ((long)g.nx * g.ny));
  return v;
}

using Set = std::vector<uint8_t>;  // byte per voxel

// Forward sets: F_0 = {root} if free; F_k = every q reachable from some
// p in F_{k-1} by an admissible, obstacle-free segment k (scatter form).
static std::vector<Set> forward_sets(const Problem& P, const V3& root) {
  const Grid& g = P.g;
  std::vector<Set> F(P.S() + 1, Set(g.nvox(), 0));
  if (g.inside(root.x, root.y, root.z) && !P.occ[g.index(root.x, root.y, root.z)])
    F[0][g.index(root.x, root.y, root.z)] = 1;
  for (int k = 1; k <= P.S(); ++k) {
    const Segment& s = P.seg[k - 1];
    for (long i = 0; i < g.nvox(); ++i) {
      if (!F[k - 1][i]) continue;
      V3 p = at(g, i);
      for (size_t e = 0; e < s.offs.size(); ++e) {
        V3 q{p.x + s.offs[e].x, p.y + s.offs[e].y, p.z + s.offs[e].z};
        if (!g.inside(q.x, q.y, q.z)) continue;
        long qi = g.index(q.x, q.y, q.z);
        if (F[k][qi]) continue;  // already known reachable
        if (edge_free(P, p, s.sc[e])) F[k][qi] = 1;
      }
    }
  }
  return F;
}

// Backward sets from a target set T: B_S = T & free; B_{k-1} = every p from
// which an admissible, obstacle-free segment k lands in B_k (mirror scatter).
// These are NOT masked by F: V_k = F_k & B_k is formed afterwards.
static std::vector<Set> backward_sets(const Problem& P, const Set& T) {
  const Grid& g = P.g;
  const int S = P.S();
  std::vector<Set> B(S + 1, Set(g.nvox(), 0));
  for (long i = 0; i < g.nvox(); ++i) B[S][i] = (T[i] && !P.occ[i]) ? 1 : 0;
  for (int k = S; k >= 1; --k) {
    const Segment& s = P.seg[k - 1];
    for (long i = 0; i < g.nvox(); ++i) {
      if (!B[k][i]) continue;
      V3 q = at(g, i);
      for (size_t e = 0; e < s.offs.size(); ++e) {
        V3 p{q.x - s.offs[e].x, q.y - s.offs[e].y, q.z - s.offs[e].z};
        if (!g.inside(p.x, p.y, p.z)) continue;
        long pi = g.index(p.x, p.y, p.z);
        if (B[k - 1][pi]) continue;
        if (edge_free(P, p, s.sc[e])) B[k - 1][pi] = 1;
      }
    }
  }
  return B;
}

static std::vector<Set> intersect(const std::vector<Set>& F, const std::vector<Set>& B) {
  std::vector<Set> V(F.size());
  for (size_t k = 0; k < F.size(); ++k) {
    V[k].resize(F[k].size());
    for (size_t i = 0; i < F[k].size(); ++i) V[k][i] = (F[k][i] && B[k][i]) ? 1 : 0;
  }
  return V;
}

// Reach traceback (Step 3 picks one surviving chain): p_0 = root; for k = 1..S, p_k is the
// voxel of V_k with the smallest linear index among those reachable from
// p_{k-1} by an admissible, obstacle-free segment k.  Returns false when
// V_0 is empty.
static bool traceback_min_index(const Problem& P, const std::vector<Set>& V, const V3& root,
                                std::vector<V3>* pose) {
  const Grid& g = P.g;
  if (!g.inside(root.x, root.y, root.z) || !V[0][g.index(root.x, root.y, root.z)]) return false;
  pose->assign(P.S() + 1, V3{0, 0, 0});
  (*pose)[0] = root;
  for (int k = 1; k <= P.S(); ++k) {
    const Segment& s = P.seg[k - 1];
    const V3 p = (*pose)[k - 1];
    long best = -1;
    for (size_t e = 0; e < s.offs.size(); ++e) {
      V3 q{p.x + s.offs[e].x, p.y + s.offs[e].y, p.z + s.offs[e].z};
      if (!g.inside(q.x, q.y, q.z)) continue;
      long qi = g.index(q.x, q.y, q.z);
      if (!V[k][qi]) continue;
      if (!edge_free(P, p, s.sc[e])) continue;
      if (best < 0 || qi < best) best = qi;
    }
    if (best < 0) return false;  // cannot happen when V_0 is non-empty
    (*pose)[k] = at(g, best);
  }
  return true;
}

static bool any(const Set& s) {
  for (uint8_t v : s)
    if (v) return true;
  return false;
}

// ---------------------------------------------------------------------------
// Path planning
// ---------------------------------------------------------------------------

// Guide waypoints on the reach polyline by the nominal arc parameter: the
// collision sample points of section "Path Planning" become W points spaced
// evenly in nominal length Lambda = sum L_k.  Waypoint j sits on segment k
// with C_{k-1} <= j*Lambda/(W-1) < C_k (the last one on segment S), at
// fraction r/den = (j*Lambda - C_{k-1}(W-1)) / (L_k (W-1)) of the segment,
// rounded half up per component: g = p_{k-1} + floor((2 r D + den) / (2 den)).
static long floor_div(long a, long b) {  // b > 0
  long q = a / b;
  if ((a % b != 0) && (a < 0)) --q;
  return q;
}

static std::vector<V3> guide_points(const std::vector<int>& L, const std::vector<V3>& pose, int W) {
  const int S = (int)L.size();
  long Lam = 0;
  for (int v : L) Lam += v;
  std::vector<long> C(S + 1, 0);
  for (int k = 1; k <= S; ++k) C[k] = C[k - 1] + L[k - 1];
  std::vector<V3> g(W);
  for (int j = 0; j < W; ++j) {
    long num = (long)j * Lam;  // s_j * (W - 1)
    int k = S;
    for (int kk = 1; kk <= S; ++kk) {
      if (C[kk - 1] * (W - 1) <= num && num < C[kk] * (W - 1)) {
        k = kk;
        break;
      }
    }
    long r = num - C[k - 1] * (W - 1);
    long den = (long)L[k - 1] * (W - 1);
    const V3& a = pose[k - 1];
    const V3& b = pose[k];
    long D[3] = {b.x - a.x, b.y - a.y, b.z - a.z};
    long o[3];
    for (int i = 0; i < 3; ++i) o[i] = floor_div(2 * r * D[i] + den, 2 * den);
    g[j] = V3{a.x + (int)o[0], a.y + (int)o[1], a.z + (int)o[2]};
  }
  return g;
}

// Guide points of a follower on joint F (section "Path Planning": the n
// collision sample points along each segment double as the waypoints): n
// points per segment of the reach polyline p_0 .. p_F, the i-th point of
// segment k at p_{k-1} + (i/n)(p_k - p_{k-1}) rounded half up per
// component, i = 0 .. n-1, and a last point p_F.  W = F n + 1.
static std::vector<V3> guide_points_per_segment(const std::vector<V3>& pose, int F, int n) {
  std::vector<V3> g(F * n + 1);
  for (int k = 1; k <= F; ++k) {
    const V3& a = pose[k - 1];
    const V3& b = pose[k];
    const long D[3] = {b.x - a.x, b.y - a.y, b.z - a.z};
    for (int i = 0; i < n; ++i) {
      long o[3];
      for (int c = 0; c < 3; ++c) o[c] = floor_div(2L * i * D[c] + n, 2L * n);
      g[(k - 1) * n + i] = V3{a.x + (int)o[0], a.y + (int)o[1], a.z + (int)o[2]};
    }
  }
  g[F * n] = pose[F];
  return g;
}

// Where the folded last segment points at waypoint j (section "Path
// Planning": the segment beyond the follower is kept clear of obstacles by
// laying it along the path the reach pose defines).  Guide point j sits at
// nominal arc length s_j = C_{k-1} + (i/n) L_k on the polyline p_0 .. p_S
// (C_k = L_1 + ... + L_k); the point aimed at is the one at arc length
// s_j + L_S, on the segment k' with C_{k'-1} <= s_j + L_S < C_{k'} (the last
// segment when s_j + L_S = C_S), as the exact rational A / den.
static void fold_point(const std::vector<int>& L, const std::vector<V3>& pose, int F, int n, int j,
                       long A[3], long* den) {
  int k = j / n + 1, i = j - (k - 1) * n;
  if (k > F) {
    k = F;
    i = n;
  }
  const int S = F + 1;
  std::vector<long> C(S + 1, 0);
  for (int q = 1; q <= S; ++q) C[q] = C[q - 1] + L[q - 1];
  const long T = (long)n * C[k - 1] + (long)i * L[k - 1] + (long)n * L[S - 1];  // n (s_j + L_S)
  int kk = S;
  for (int q = 1; q <= S; ++q)
    if ((long)n * C[q - 1] <= T && T < (long)n * C[q]) {
      kk = q;
      break;
    }
  *den = (long)n * L[kk - 1];
  const long num = T - (long)n * C[kk - 1];
  const V3& a = pose[kk - 1];
  const V3& b = pose[kk];
  A[0] = *den * a.x + num * (b.x - a.x);
  A[1] = *den * a.y + num * (b.y - a.y);
  A[2] = *den * a.z + num * (b.z - a.z);
}

// The folded last segment from the follower f: among the admissible,
// obstacle-free segments S from f that end inside the grid, the end
// nearest to A / den (squared distance), then the smallest linear index.
static bool fold_end(const Problem& P, const V3& f, const long A[3], long den, V3* out) {
  const Grid& g = P.g;
  const Segment& s = P.seg[P.S() - 1];
  bool found = false;
  long best = 0, best_i = 0;
  for (size_t e = 0; e < s.offs.size(); ++e) {
    const V3 q{f.x + s.offs[e].x, f.y + s.offs[e].y, f.z + s.offs[e].z};
    if (!g.inside(q.x, q.y, q.z)) continue;
    if (!edge_free(P, f, s.sc[e])) continue;
    const long key = sq(den * q.x - A[0]) + sq(den * q.y - A[1]) + sq(den * q.z - A[2]);
    const long qi = g.index(q.x, q.y, q.z);
    if (!found || key < best || (key == best && qi < best_i)) {
      found = true;
      best = key;
      best_i = qi;
      *out = q;
    }
  }
  return found;
}

// Waypoint target set: free voxels within squared distance eps2 of g.  When
// it is empty the radius grows one unit of eps2 at a time up to eps2_max.
static Set waypoint_target(const Problem& P, const V3& gpt, int eps2, int eps2_max, int* used) {
  const Grid& g = P.g;
  Set T(g.nvox(), 0);
  for (int e2 = eps2; e2 <= std::max(eps2, eps2_max); ++e2) {
    bool found = false;
    int R = 0;
    while ((R + 1) * (R + 1) <= e2) ++R;
    for (int z = gpt.z - R; z <= gpt.z + R; ++z)
      for (int y = gpt.y - R; y <= gpt.y + R; ++y)
        for (int x = gpt.x - R; x <= gpt.x + R; ++x) {
          if (!g.inside(x, y, z)) continue;
          if (dist2(V3{x, y, z}, gpt) > e2) continue;
          long i = g.index(x, y, z);
          if (P.occ[i]) continue;
          T[i] = 1;
          found = true;
        }
    if (found) {
      *used = e2;
      return T;
    }
  }
  *used = -1;
  return T;
}

// One smooth-chain step (section "Smooth sequence computation": the pose
// nearest in configuration to the previous one; section "Filtering for
// smoothness"): with joint k restricted to
// C_k = V_k & Ball(ref_k, r_k) (r2[k] = r_k^2; r2[k] < 0: joint k is not
// filtered, C_k = V_k), find the chains root -> ... -> end in V_S, by
// forward restriction then backward restriction, and take the
// minimum-linear-index traceback.  Returns false when no chain fits.
static bool smooth_step_radii(const Problem& P, const std::vector<Set>& V, const std::vector<V3>& ref,
                              const std::vector<long>& r2, std::vector<V3>* pose) {
  const Grid& g = P.g;
  const int S = P.S();
  auto in_ball = [&](int k, long i) { return r2[k] < 0 || dist2(at(g, i), ref[k]) <= r2[k]; };
  const V3 root = ref[0];
  long root_i = g.index(root.x, root.y, root.z);
  if (!V[0][root_i]) return false;
  // forward restriction
  std::vector<std::vector<long>> R(S + 1);
  std::vector<Set> Rm(S + 1, Set(g.nvox(), 0));
  R[0].push_back(root_i);
  Rm[0][root_i] = 1;
  for (int k = 1; k <= S; ++k) {
    const Segment& s = P.seg[k - 1];
    for (long pi : R[k - 1]) {
      V3 p = at(g, pi);
      for (size_t e = 0; e < s.offs.size(); ++e) {
        V3 q{p.x + s.offs[e].x, p.y + s.offs[e].y, p.z + s.offs[e].z};
        if (!g.inside(q.x, q.y, q.z)) continue;
        long qi = g.index(q.x, q.y, q.z);
        if (Rm[k][qi] || !V[k][qi] || !in_ball(k, qi)) continue;
        if (!edge_free(P, p, s.sc[e])) continue;
        Rm[k][qi] = 1;
        R[k].push_back(qi);
      }
    }
    if (R[k].empty()) return false;
  }
  // backward restriction
  std::vector<Set> U(S + 1, Set(g.nvox(), 0));
  for (long qi : R[S]) U[S][qi] = 1;
  for (int k = S - 1; k >= 0; --k) {
    const Segment& s = P.seg[k];
    for (long pi : R[k]) {
      V3 p = at(g, pi);
      for (size_t e = 0; e < s.offs.size(); ++e) {
        V3 q{p.x + s.offs[e].x, p.y + s.offs[e].y, p.z + s.offs[e].z};
        if (!g.inside(q.x, q.y, q.z)) continue;
        if (!U[k + 1][g.index(q.x, q.y, q.z)]) continue;
        if (!edge_free(P, p, s.sc[e])) continue;
        U[k][pi] = 1;
        break;
      }
    }
  }
  if (!U[0][root_i]) return false;
  return traceback_min_index(P, U, root, pose);
}

// Every joint within delta of its reference.
static bool smooth_step(const Problem& P, const std::vector<Set>& V, const std::vector<V3>& ref,
                        long delta, std::vector<V3>* pose) {
  return smooth_step_radii(P, V, ref, std::vector<long>(P.S() + 1, delta * delta), pose);
}

static bool pose_valid(const Problem& P, const std::vector<V3>& pose) {
  const Grid& g = P.g;
  for (int k = 0; k <= P.S(); ++k)
    if (!g.inside(pose[k].x, pose[k].y, pose[k].z)) return false;
  for (int k = 1; k <= P.S(); ++k) {
    V3 d{pose[k].x - pose[k - 1].x, pose[k].y - pose[k - 1].y, pose[k].z - pose[k - 1].z};
    if (!is_offset_in_shell(P.seg[k - 1], d)) return false;
    for (const V3& v : supercover(pose[k - 1], pose[k]))
      if (P.occ[g.index(v.x, v.y, v.z)]) return false;
  }
  return true;
}

static long diag2(const Grid& g) {
  return sq(g.nx - 1) + sq(g.ny - 1) + sq(g.nz - 1);
}

// Relaxation ladder (section "Filtering for smoothness": the filter is
// relaxed only after a waypoint fails): delta, delta+1, ... until a chain is found or the ball
// covers the whole grid (delta^2 >= squared grid diagonal), or max_relax
// increments have been tried (max_relax < 0: no cap).  Returns the number
// of increments used, or -1.
static int smooth_ladder(const Problem& P, const std::vector<Set>& V, const std::vector<V3>& ref,
                         int delta, int max_relax, std::vector<V3>* pose) {
  if (!any(V[0])) return -1;
  const long D2 = diag2(P.g);
  for (int m = 0;; ++m) {
    if (max_relax >= 0 && m > max_relax) return -1;
    long d = (long)delta + m;
    if (smooth_step(P, V, ref, d, pose)) return m;
    if (d * d >= D2) return -1;
  }
}

// The same ladder with a radius per joint (rad[k] for joint k = 1..S, -1:
// joint k is not filtered): try rad[k] + m for m = 0, 1, ... until a chain
// is found, or every filtered joint's ball covers the grid, or max_relax
// increments have been tried.
static int smooth_ladder_radii(const Problem& P, const std::vector<Set>& V, const std::vector<V3>& ref,
                               const std::vector<int>& rad, int max_relax, std::vector<V3>* pose) {
  if (!any(V[0])) return -1;
  const long D2 = diag2(P.g);
  const int S = P.S();
  for (int m = 0;; ++m) {
    if (max_relax >= 0 && m > max_relax) return -1;
    std::vector<long> r2(S + 1, -1);
    bool covered = true;
    for (int k = 1; k <= S; ++k) {
      if (rad[k] < 0) continue;
      const long r = (long)rad[k] + m;
      r2[k] = r * r;
      if (r * r < D2) covered = false;
    }
    if (smooth_step_radii(P, V, ref, r2, pose)) return m;
    if (covered) return -1;
  }
}

enum { PATH_OK = 0, PATH_RELAXED = 1, PATH_BROKEN = 2, PATH_UNREACHABLE = 3, PATH_KEPT = 4 };

struct PathParams {
  int W, delta, eps2, eps2_max, max_relax;
};

static std::vector<Set> waypoint_V(const Problem& P, const std::vector<Set>& F, const Set& T) {
  return intersect(F, backward_sets(P, T));
}

// Approach cone on the last segment (section "The gap in gMS": the backward
// search from the target starts from the directions the last segment may
// arrive along, one vector or a cone of them).  cone = {ax, ay, az, num,
// den}: the segment vector s (from joint S-1 to the end effector) is
// admissible when it points into the half-space of the axis a and its angle
// to a is at most theta with cos^2 theta = num / den, i.e.
//   s.a > 0  and  den * (s.a)^2 >= num * |s|^2 * |a|^2   (exact integers).
static bool in_cone(const V3& s, const int32_t* c) {
  const long dot = (long)s.x * c[0] + (long)s.y * c[1] + (long)s.z * c[2];
  if (dot <= 0) return false;
  const long s2 = sq(s.x) + sq(s.y) + sq(s.z);
  const long a2 = sq(c[0]) + sq(c[1]) + sq(c[2]);
  return (long)c[4] * dot * dot >= (long)c[3] * s2 * a2;
}

// The offsets of segment s (with their supercovers) that lie in the cone.
static Segment cone_segment(const Segment& s, const int32_t* c) {
  Segment out;
  out.lo2 = s.lo2;
  out.hi2 = s.hi2;
  for (size_t i = 0; i < s.offs.size(); ++i) {
    if (!in_cone(s.offs[i], c)) continue;
    out.offs.push_back(s.offs[i]);
    out.sc.push_back(s.sc[i]);
  }
  return out;
}

// limits (nullable) [S][5]: per-segment direction limits (section "The
// procedure for IK solution", Step 1 (a): joint 1 angle constraints, e.g. the
// first segment restricted to the upper hemisphere, section "The gap in
// gMS").  Row k = {ax, ay, az, num, den} keeps the offsets of segment k+1 in
// that cone (the same test as in_cone); an all-zero axis leaves it whole.
static Problem make_problem(int nx, int ny, int nz, const uint8_t* occ, int S, const int32_t* lo2,
                            const int32_t* hi2, const int32_t* limits = nullptr) {
  Problem P;
  P.g = Grid{nx, ny, nz};
  P.occ = occ;
  for (int k = 0; k < S; ++k) {
    Segment s = make_segment(lo2[k], hi2[k]);
    const int32_t* c = limits ? limits + 5 * k : nullptr;
    if (c && (c[0] != 0 || c[1] != 0 || c[2] != 0)) s = cone_segment(s, c);
    P.seg.push_back(s);
  }
  return P;
}

static std::vector<V3> read_pose(const int32_t* p, int S) {
  std::vector<V3> v(S + 1);
  for (int k = 0; k <= S; ++k) v[k] = V3{p[3 * k], p[3 * k + 1], p[3 * k + 2]};
  return v;
}
static void write_pose(const std::vector<V3>& v, int32_t* p) {
  for (size_t k = 0; k < v.size(); ++k) {
    p[3 * k] = v[k].x;
    p[3 * k + 1] = v[k].y;
    p[3 * k + 2] = v[k].z;
  }
}

}  // namespace

extern "C" {

int orc_shell_bounds(int L, double tol, int* lo2, int* hi2) {
  shell_bounds(L, tol, lo2, hi2);
  return 0;
}

// Writes up to cap offsets (x,y,z int32 triples); returns the shell size.
int orc_shell(int lo2, int hi2, int32_t* out, int cap) {
  std::vector<V3> s = shell(lo2, hi2);
  for (int i = 0; i < (int)s.size() && i < cap; ++i) {
    out[3 * i] = s[i].x;
    out[3 * i + 1] = s[i].y;
    out[3 * i + 2] = s[i].z;
  }
  return (int)s.size();
}

// Supercover of a->b in (z,y,x) order; returns its size.
int orc_supercover(const int32_t* a, const int32_t* b, int32_t* out, int cap) {
  std::vector<V3> s = supercover(V3{a[0], a[1], a[2]}, V3{b[0], b[1], b[2]});
  for (int i = 0; i < (int)s.size() && i < cap; ++i) {
    out[3 * i] = s[i].x;
    out[3 * i + 1] = s[i].y;
    out[3 * i + 2] = s[i].z;
  }
  return (int)s.size();
}

// Occupancy from inclusive boxes (lo_xyz, hi_xyz), clipped to the grid.
int orc_rasterize(int nx, int ny, int nz, const int32_t* boxes, int nbox, uint8_t* occ) {
  Grid g{nx, ny, nz};
  std::memset(occ, 0, (size_t)g.nvox());
  for (int b = 0; b < nbox; ++b) {
    const int32_t* B = boxes + 6 * b;
    for (int z = std::max(0, B[2]); z <= std::min(nz - 1, B[5]); ++z)
      for (int y = std::max(0, B[1]); y <= std::min(ny - 1, B[4]); ++y)
        for (int x = std::max(0, B[0]); x <= std::min(nx - 1, B[3]); ++x) occ[g.index(x, y, z)] = 1;
  }
  return 0;
}

// F_0..F_S as bytes, [(S+1)][nvox].
int orc_forward(int nx, int ny, int nz, const uint8_t* occ, int S, const int32_t* lo2,
                const int32_t* hi2, const int32_t* root, uint8_t* fsets, const int32_t* limits) {
  Problem P = make_problem(nx, ny, nz, occ, S, lo2, hi2, limits);
  std::vector<Set> F = forward_sets(P, V3{root[0], root[1], root[2]});
  for (int k = 0; k <= S; ++k) std::memcpy(fsets + (size_t)k * P.g.nvox(), F[k].data(), P.g.nvox());
  return 0;
}

// Unmasked backward sets B_0..B_S from a target set T (bytes).
int orc_backward(int nx, int ny, int nz, const uint8_t* occ, int S, const int32_t* lo2,
                 const int32_t* hi2, const uint8_t* T, uint8_t* bsets) {
  Problem P = make_problem(nx, ny, nz, occ, S, lo2, hi2);
  Set t(T, T + P.g.nvox());
  std::vector<Set> B = backward_sets(P, t);
  for (int k = 0; k <= S; ++k) std::memcpy(bsets + (size_t)k * P.g.nvox(), B[k].data(), P.g.nvox());
  return 0;
}

// Reach for many point targets sharing one root: F once, then per target
// B, V = F & B and the traceback.  poses_out [n][S+1][3], found_out [n],
// vsets_out (nullable) [n][S+1][nvox].  Targets are split across n_threads.
int orc_reach_many(int nx, int ny, int nz, const uint8_t* occ, int S, const int32_t* lo2,
                   const int32_t* hi2, const int32_t* root, int n, const int32_t* targets,
                   int32_t* poses_out, int32_t* found_out, uint8_t* vsets_out, int n_threads,
                   const int32_t* limits) {
  Problem P = make_problem(nx, ny, nz, occ, S, lo2, hi2, limits);
  const V3 r{root[0], root[1], root[2]};
  std::vector<Set> F = forward_sets(P, r);
  auto work = [&](int t0, int step) {
    for (int t = t0; t < n; t += step) {
      Set T(P.g.nvox(), 0);
      V3 tv{targets[3 * t], targets[3 * t + 1], targets[3 * t + 2]};
      if (P.g.inside(tv.x, tv.y, tv.z)) T[P.g.index(tv.x, tv.y, tv.z)] = 1;
      std::vector<Set> V = intersect(F, backward_sets(P, T));
      std::vector<V3> pose;
      bool ok = traceback_min_index(P, V, r, &pose);
      found_out[t] = ok ? 1 : 0;
      if (!ok) pose.assign(S + 1, V3{0, 0, 0});
      write_pose(pose, poses_out + (size_t)t * 3 * (S + 1));
      if (vsets_out)
        for (int k = 0; k <= S; ++k)
          std::memcpy(vsets_out + ((size_t)t * (S + 1) + k) * P.g.nvox(), V[k].data(), P.g.nvox());
    }
  };
  if (n_threads <= 1) {
    work(0, 1);
  } else {
    std::vector<std::thread> th;
    for (int i = 0; i < n_threads; ++i) th.emplace_back(work, i, n_threads);
    for (auto& x : th) x.join();
  }
  return 0;
}

// Reach for a target set T (bytes [nvox]; a cloud of targets,
// section "Dynamic Obstacles") with an optional approach cone on the last
// segment (nullptr: any direction).  F is grown with the full shells; the
// backward sets from T and the traceback use segment S restricted to the
// cone, so every found chain ends in T with its last segment in the cone.
// V_S keeps its definition F_S & T.  pose_out [S+1][3]; vsets_out
// (nullable) [S+1][nvox]; *found_out 1 / 0.
int orc_reach_set(int nx, int ny, int nz, const uint8_t* occ, int S, const int32_t* lo2,
                  const int32_t* hi2, const int32_t* root, const uint8_t* T, const int32_t* cone,
                  int32_t* pose_out, uint8_t* vsets_out, int32_t* found_out) {
  Problem P = make_problem(nx, ny, nz, occ, S, lo2, hi2);
  const V3 r{root[0], root[1], root[2]};
  std::vector<Set> F = forward_sets(P, r);
  Problem Pc = P;
  if (cone) Pc.seg[S - 1] = cone_segment(P.seg[S - 1], cone);
  Set t(T, T + P.g.nvox());
  std::vector<Set> V = intersect(F, backward_sets(Pc, t));
  std::vector<V3> pose;
  const bool ok = traceback_min_index(Pc, V, r, &pose);
  *found_out = ok ? 1 : 0;
  if (!ok) pose.assign(S + 1, V3{0, 0, 0});
  write_pose(pose, pose_out);
  if (vsets_out)
    for (int k = 0; k <= S; ++k) std::memcpy(vsets_out + (size_t)k * P.g.nvox(), V[k].data(), P.g.nvox());
  return 0;
}

// Path between arbitrary poses (section "Path between Arbitrary Poses"): a
// virtual arm (Sv segments, shells vlo2/vhi2, nominal lengths vlens) rooted
// at the end effector of the start pose reaches for the target with the
// reach search (F, B, V = F & B, minimum-index traceback); its pose is the
// guide polyline of the end effector (guide points by the nominal-arc rule of
// the virtual arm, g_0 = the start's end effector, g_{W-1} = the target).
// The actual arm's pose^(0) is the start pose and poses 1..W-1 are chained
// forward, each the smooth step around the previous pose with its
// relaxation ladder, waypoint targets as for any path (T_{W-1} = {target}).
// No valid start pose, target outside the grid or no virtual reach:
// PATH_UNREACHABLE, every pose the start pose, relax m = -1 for j >= 1.
// poses_out [W][S+1][3], relax_out [W][2], vpose_out (nullable) [Sv+1][3].
int orc_plan_between(int nx, int ny, int nz, const uint8_t* occ, int S, const int32_t* lo2,
                     const int32_t* hi2, const int32_t* start_pose, int Sv, const int32_t* vlens,
                     const int32_t* vlo2, const int32_t* vhi2, const int32_t* target, int W, int delta,
                     int eps2, int eps2_max, int max_relax, int32_t* poses_out, int32_t* relax_out,
                     int32_t* status_out, int32_t* vpose_out) {
  Problem P = make_problem(nx, ny, nz, occ, S, lo2, hi2);
  Problem Pv = make_problem(nx, ny, nz, occ, Sv, vlo2, vhi2);
  const std::vector<V3> start = read_pose(start_pose, S);
  std::vector<std::vector<V3>> poses(W, start);
  for (int j = 0; j < W; ++j) relax_out[2 * j] = relax_out[2 * j + 1] = 0;
  const V3 t{target[0], target[1], target[2]};
  auto unreachable = [&]() {
    for (int j = 1; j < W; ++j) relax_out[2 * j] = -1;
    for (int j = 0; j < W; ++j) write_pose(poses[j], poses_out + (size_t)j * 3 * (S + 1));
    *status_out = PATH_UNREACHABLE;
    return 0;
  };
  if (W < 2 || !pose_valid(P, start) || !P.g.inside(t.x, t.y, t.z)) return unreachable();
  // the virtual arm's reach from the start's end effector
  const V3 vroot = start[S];
  Set T(P.g.nvox(), 0);
  T[P.g.index(t.x, t.y, t.z)] = 1;
  std::vector<Set> Vv = intersect(forward_sets(Pv, vroot), backward_sets(Pv, T));
  std::vector<V3> vpose;
  if (!traceback_min_index(Pv, Vv, vroot, &vpose)) return unreachable();
  if (vpose_out) write_pose(vpose, vpose_out);
  std::vector<int> Lv(vlens, vlens + Sv);
  const std::vector<V3> g = guide_points(Lv, vpose, W);
  // the actual arm, chained forward from the start pose
  std::vector<Set> F = forward_sets(P, start[0]);
  bool relaxed = false, broken = false;
  for (int j = 1; j < W; ++j) {
    int used = 0;
    Set Tj;
    if (j == W - 1) {
      Tj = T;
    } else {
      Tj = waypoint_target(P, g[j], eps2, eps2_max, &used);
      if (used != eps2) relaxed = true;
    }
    std::vector<Set> V = waypoint_V(P, F, Tj);
    std::vector<V3> pose;
    const int m = smooth_ladder(P, V, poses[j - 1], delta, max_relax, &pose);
    relax_out[2 * j + 1] = used;
    if (m < 0) {
      broken = true;
      poses[j] = poses[j - 1];
      relax_out[2 * j] = -1;
    } else {
      if (m > 0) relaxed = true;
      poses[j] = pose;
      relax_out[2 * j] = m;
    }
  }
  for (int j = 0; j < W; ++j) write_pose(poses[j], poses_out + (size_t)j * 3 * (S + 1));
  *status_out = broken ? PATH_BROKEN : (relaxed ? PATH_RELAXED : PATH_OK);
  return 0;
}

// Obstacle dilation (section "Testing for collisions": the obstacle volumes
// are dilated when the grid is initialised, to account for the thickness of
// the arm and a clearance margin): out[p] = 1 when some occupied voxel q has
// |p - q|^2 <= r2.  A plain scatter over the occupied voxels and every
// integer offset of the ball.
int orc_dilate(int nx, int ny, int nz, const uint8_t* occ, int r2, uint8_t* out) {
  Grid g{nx, ny, nz};
  std::memset(out, 0, (size_t)g.nvox());
  int r = 0;
  while ((long)(r + 1) * (r + 1) <= r2) ++r;
  for (long i = 0; i < g.nvox(); ++i) {
    if (!occ[i]) continue;
    const V3 q = at(g, i);
    for (int dz = -r; dz <= r; ++dz)
      for (int dy = -r; dy <= r; ++dy)
        for (int dx = -r; dx <= r; ++dx) {
          if ((long)dx * dx + (long)dy * dy + (long)dz * dz > r2) continue;
          const int x = q.x + dx, y = q.y + dy, z = q.z + dz;
          if (g.inside(x, y, z)) out[g.index(x, y, z)] = 1;
        }
  }
  return 0;
}

// Pose validity: joints inside the grid, offsets in the shells, every
// supercover voxel free.  Returns 1 / 0.
int orc_pose_valid(int nx, int ny, int nz, const uint8_t* occ, int S, const int32_t* lo2,
                   const int32_t* hi2, const int32_t* pose, const int32_t* limits) {
  Problem P = make_problem(nx, ny, nz, occ, S, lo2, hi2, limits);
  return pose_valid(P, read_pose(pose, S)) ? 1 : 0;
}

int orc_guide(int S, const int32_t* lens, const int32_t* pose, int W, int32_t* g_out) {
  std::vector<int> L(lens, lens + S);
  std::vector<V3> g = guide_points(L, read_pose(pose, S), W);
  write_pose(g, g_out);
  return 0;
}

// Waypoint target sets and their survivor sets V^(j) for all j (bytes):
// T_j from the guide points (T_{W-1} = {end effector of the reach pose}),
// eps2_used [W], vsets_out [W][S+1][nvox] (nullable).
int orc_waypoint_sets(int nx, int ny, int nz, const uint8_t* occ, int S, const int32_t* lens,
                      const int32_t* lo2, const int32_t* hi2, const int32_t* reach_pose, int W,
                      int eps2, int eps2_max, int32_t* eps2_used, uint8_t* vsets_out, int n_threads) {
  Problem P = make_problem(nx, ny, nz, occ, S, lo2, hi2);
  std::vector<V3> reach = read_pose(reach_pose, S);
  std::vector<int> L(lens, lens + S);
  std::vector<V3> g = guide_points(L, reach, W);
  std::vector<Set> F = forward_sets(P, reach[0]);
  auto work = [&](int t0, int step) {
    for (int j = t0; j < W; j += step) {
      Set T;
      if (j == W - 1) {
        T.assign(P.g.nvox(), 0);
        T[P.g.index(reach[S].x, reach[S].y, reach[S].z)] = 1;
        eps2_used[j] = 0;
      } else {
        T = waypoint_target(P, g[j], eps2, eps2_max, &eps2_used[j]);
      }
      std::vector<Set> V = waypoint_V(P, F, T);
      if (vsets_out)
        for (int k = 0; k <= S; ++k)
          std::memcpy(vsets_out + ((size_t)j * (S + 1) + k) * P.g.nvox(), V[k].data(), P.g.nvox());
    }
  };
  if (n_threads <= 1) {
    work(0, 1);
  } else {
    std::vector<std::thread> th;
    for (int i = 0; i < n_threads; ++i) th.emplace_back(work, i, n_threads);
    for (auto& x : th) x.join();
  }
  return 0;
}

// Path planning ("Smooth sequence computation"): pose^(W-1) = reach pose;
// for j = W-2 .. 0 the pose at waypoint j is the smooth step around
// pose^(j+1) with the relaxation ladder.  A waypoint whose survivor set is
// empty is skipped (its pose repeats pose^(j+1), record -1).
// relax_out [W][2] = {delta increments or -1, eps2 used}.
static void plan_backward(const Problem& P, const std::vector<V3>& reach, const std::vector<V3>& g, int W,
                          int delta, int eps2, int eps2_max, int max_relax, int32_t* poses_out,
                          int32_t* relax_out, int32_t* status_out);

int orc_plan_path(int nx, int ny, int nz, const uint8_t* occ, int S, const int32_t* lens,
                  const int32_t* lo2, const int32_t* hi2, const int32_t* reach_pose, int W,
                  int delta, int eps2, int eps2_max, int max_relax, int32_t* poses_out,
                  int32_t* relax_out, int32_t* status_out, const int32_t* limits) {
  Problem P = make_problem(nx, ny, nz, occ, S, lo2, hi2, limits);
  std::vector<V3> reach = read_pose(reach_pose, S);
  if (W < 2 || !pose_valid(P, reach)) {
    *status_out = PATH_UNREACHABLE;
    return -1;
  }
  std::vector<int> L(lens, lens + S);
  plan_backward(P, reach, guide_points(L, reach, W), W, delta, eps2, eps2_max, max_relax, poses_out,
                relax_out, status_out);
  return 0;
}

// Short reaches (section "Short Reaches": a near encounter of an early
// segment hypothesis with the target makes a shorter path than the reach
// pose's polyline).  For k = 1 .. kmax and, within k, l = 1 .. L_k, a virtual
// arm of the segments L_1 .. L_{k-1} and one of length l (its shell from l
// and tol, as for any segment: the shell tolerance is the encounter
// tolerance) is rooted at the root and reaches for the target with the
// reach search; the first virtual arm that reaches it has the smallest
// nominal length L_1 + ... + L_{k-1} + l, and its pose is the guide
// polyline (guide points by the nominal arc rule of its lengths).  Without
// one the reach pose's polyline is the guide.  The poses then follow
// orc_plan_path (backward from the reach pose).  shortcut_out [2] = {k, l}
// ({0, 0}: no shortcut); vpose_out (nullable) [k+1][3], the shortcut's pose.
int orc_plan_short(int nx, int ny, int nz, const uint8_t* occ, int S, const int32_t* lens,
                   const int32_t* lo2, const int32_t* hi2, double tol, const int32_t* reach_pose, int W,
                   int delta, int eps2, int eps2_max, int max_relax, int kmax, int32_t* poses_out,
                   int32_t* relax_out, int32_t* status_out, int32_t* shortcut_out, int32_t* vpose_out) {
  Problem P = make_problem(nx, ny, nz, occ, S, lo2, hi2);
  std::vector<V3> reach = read_pose(reach_pose, S);
  shortcut_out[0] = shortcut_out[1] = 0;
  if (W < 2 || !pose_valid(P, reach)) {
    *status_out = PATH_UNREACHABLE;
    return -1;
  }
  std::vector<int> L(lens, lens + S);
  const V3 root = reach[0], t = reach[S];
  Set T(P.g.nvox(), 0);
  T[P.g.index(t.x, t.y, t.z)] = 1;
  std::vector<int> glen = L;
  std::vector<V3> gpose = reach;
  bool found = false;
  for (int k = 1; k <= std::min(kmax, S) && !found; ++k) {
    for (int l = 1; l <= L[k - 1] && !found; ++l) {
      std::vector<int> vl(L.begin(), L.begin() + k), vlo(k), vhi(k);
      vl[k - 1] = l;
      for (int q = 0; q < k; ++q) shell_bounds(vl[q], tol, &vlo[q], &vhi[q]);
      Problem Pv = make_problem(nx, ny, nz, occ, k, vlo.data(), vhi.data());
      std::vector<Set> V = intersect(forward_sets(Pv, root), backward_sets(Pv, T));
      std::vector<V3> vpose;
      if (traceback_min_index(Pv, V, root, &vpose)) {
        found = true;
        glen = vl;
        gpose = vpose;
        shortcut_out[0] = k;
        shortcut_out[1] = l;
        if (vpose_out) write_pose(vpose, vpose_out);
      }
    }
  }
  plan_backward(P, reach, guide_points(glen, gpose, W), W, delta, eps2, eps2_max, max_relax, poses_out,
                relax_out, status_out);
  return 0;
}

// pose^(W-1) = reach pose; for j = W-2 .. 0 the pose at waypoint j is the
// smooth step around pose^(j+1) with the relaxation ladder, the end effector
// near guide point g[j].
static void plan_backward(const Problem& P, const std::vector<V3>& reach, const std::vector<V3>& g, int W,
                          int delta, int eps2, int eps2_max, int max_relax, int32_t* poses_out,
                          int32_t* relax_out, int32_t* status_out) {
  const int S = P.S();
  std::vector<Set> F = forward_sets(P, reach[0]);
  std::vector<std::vector<V3>> poses(W);
  poses[W - 1] = reach;
  relax_out[2 * (W - 1)] = 0;
  relax_out[2 * (W - 1) + 1] = 0;
  bool relaxed = false, broken = false;
  for (int j = W - 2; j >= 0; --j) {
    int used = -1;
    Set T = waypoint_target(P, g[j], eps2, eps2_max, &used);
    if (used != eps2) relaxed = true;
    std::vector<Set> V = waypoint_V(P, F, T);
    std::vector<V3> pose;
    int m = smooth_ladder(P, V, poses[j + 1], delta, max_relax, &pose);
    relax_out[2 * j + 1] = used;
    if (m < 0) {
      broken = true;
      poses[j] = poses[j + 1];
      relax_out[2 * j] = -1;
    } else {
      if (m > 0) relaxed = true;
      poses[j] = pose;
      relax_out[2 * j] = m;
    }
  }
  for (int j = 0; j < W; ++j) write_pose(poses[j], poses_out + (size_t)j * 3 * (S + 1));
  *status_out = broken ? PATH_BROKEN : (relaxed ? PATH_RELAXED : PATH_OK);
}

// Path with the paper's follower and filter (sections "Path Planning" and
// "Filtering for smoothness"): the follower is joint F = S - fold (fold = 1:
// the distal end of segment S-1, the last segment folded along the path;
// fold = 0: the end effector); it visits n guide points per segment of the
// reach polyline p_0 .. p_F, each waypoint an IK solution of the arm's first
// F segments with the follower within squared distance eps2 of the guide
// point (growing to eps2_max when no free voxel is that close; the last
// waypoint is p_F itself).  Backward from the reach pose, the pose at
// waypoint j is the smooth step around pose^(j+1) in which joint k
// (1..F) moves at most rad[k-1] voxels (rad[k-1] < 0: joint k is not
// filtered), every radius growing by one voxel at a time on failure.  With
// fold = 1 each pose's last joint is then fold_end from its follower
// towards fold_point; a pose whose last segment finds no free end keeps
// the follower's position there, records -1 and breaks the path.  A
// waypoint with no chain repeats pose^(j+1) and records -1.
// poses_out [W][S+1][3], relax_out [W][2] = {radius increments or -1, eps2
// used}; returns W = F n + 1, or -1 when the reach pose is not valid.
int orc_plan_path_follow(int nx, int ny, int nz, const uint8_t* occ, int S, const int32_t* lens,
                         const int32_t* lo2, const int32_t* hi2, const int32_t* reach_pose, int n,
                         int fold, const int32_t* rad, int eps2, int eps2_max, int max_relax,
                         int32_t* poses_out, int32_t* relax_out, int32_t* status_out) {
  Problem P = make_problem(nx, ny, nz, occ, S, lo2, hi2);
  std::vector<V3> reach = read_pose(reach_pose, S);
  const int F = S - (fold ? 1 : 0);
  if (n < 1 || F < 1 || !pose_valid(P, reach)) {
    *status_out = PATH_UNREACHABLE;
    return -1;
  }
  Problem PF = make_problem(nx, ny, nz, occ, F, lo2, hi2);
  std::vector<int> L(lens, lens + S);
  std::vector<int> radk(F + 1, -1);
  for (int k = 1; k <= F; ++k) radk[k] = rad[k - 1];
  const int W = F * n + 1;
  std::vector<V3> g = guide_points_per_segment(reach, F, n);
  std::vector<Set> Fs = forward_sets(PF, reach[0]);
  std::vector<std::vector<V3>> tp(W);  // joints 0 .. F
  tp[W - 1] = std::vector<V3>(reach.begin(), reach.begin() + F + 1);
  relax_out[2 * (W - 1)] = 0;
  relax_out[2 * (W - 1) + 1] = 0;
  bool relaxed = false, broken = false;
  for (int j = W - 2; j >= 0; --j) {
    int used = -1;
    Set T = waypoint_target(PF, g[j], eps2, eps2_max, &used);
    if (used != eps2) relaxed = true;
    std::vector<Set> V = waypoint_V(PF, Fs, T);
    std::vector<V3> pose;
    const int m = smooth_ladder_radii(PF, V, tp[j + 1], radk, max_relax, &pose);
    relax_out[2 * j + 1] = used;
    if (m < 0) {
      broken = true;
      tp[j] = tp[j + 1];
      relax_out[2 * j] = -1;
    } else {
      if (m > 0) relaxed = true;
      tp[j] = pose;
      relax_out[2 * j] = m;
    }
  }
  for (int j = 0; j < W; ++j) {
    std::vector<V3> full = tp[j];
    if (fold) {
      long A[3], den;
      fold_point(L, reach, F, n, j, A, &den);
      V3 q;
      if (fold_end(P, tp[j][F], A, den, &q)) {
        full.push_back(q);
      } else {
        full.push_back(tp[j][F]);
        relax_out[2 * j] = -1;
        broken = true;
      }
    }
    write_pose(full, poses_out + (size_t)j * 3 * (S + 1));
  }
  *status_out = broken ? PATH_BROKEN : (relaxed ? PATH_RELAXED : PATH_OK);
  return W;
}

// Midcourse replan ("Dynamic Obstacles"), given the current occupancy:
//  1. if every pose after the current index c is still valid, keep the path;
//  2. else keep the reach pose if it is still valid, or re-solve it joint by
//     joint from the root taking the successor in V_k closest to the old
//     joint (squared distance, then linear index) -- the "least distance to
//     the original path" objective applied to the reach pose that guides
//     the path;
//  3. guide points from that reach pose, survivor sets for j > c, and a
//     forward smooth chain j = c+1 .. W-1 starting from pose^(c).
int orc_replan(int nx, int ny, int nz, const uint8_t* occ, int S, const int32_t* lens,
               const int32_t* lo2, const int32_t* hi2, const int32_t* poses_in, int W, int c,
               int delta, int eps2, int eps2_max, int max_relax, int32_t* poses_out,
               int32_t* relax_out, int32_t* status_out) {
  Problem P = make_problem(nx, ny, nz, occ, S, lo2, hi2);
  std::vector<std::vector<V3>> old(W), poses(W);
  for (int j = 0; j < W; ++j) old[j] = read_pose(poses_in + (size_t)j * 3 * (S + 1), S);
  for (int j = 0; j < W; ++j) {
    relax_out[2 * j] = 0;
    relax_out[2 * j + 1] = 0;
  }
  bool cut = false;
  for (int j = c + 1; j < W; ++j)
    if (!pose_valid(P, old[j])) cut = true;
  if (!cut) {
    for (int j = 0; j < W; ++j) write_pose(old[j], poses_out + (size_t)j * 3 * (S + 1));
    *status_out = PATH_KEPT;
    return 0;
  }
  for (int j = 0; j <= c; ++j) poses[j] = old[j];
  const V3 root = old[0][0];
  std::vector<Set> F = forward_sets(P, root);
  std::vector<V3> reach = old[W - 1];
  if (!pose_valid(P, reach)) {
    Set T(P.g.nvox(), 0);
    const V3 t = old[W - 1][S];
    T[P.g.index(t.x, t.y, t.z)] = 1;
    std::vector<Set> V = intersect(F, backward_sets(P, T));
    bool ok = V[0][P.g.index(root.x, root.y, root.z)] != 0;
    if (ok) {
      reach.assign(S + 1, V3{0, 0, 0});
      reach[0] = root;
      for (int k = 1; k <= S; ++k) {
        const Segment& s = P.seg[k - 1];
        const V3 p = reach[k - 1];
        long best = -1, best_d = 0;
        for (size_t e = 0; e < s.offs.size(); ++e) {
          V3 q{p.x + s.offs[e].x, p.y + s.offs[e].y, p.z + s.offs[e].z};
          if (!P.g.inside(q.x, q.y, q.z)) continue;
          long qi = P.g.index(q.x, q.y, q.z);
          if (!V[k][qi] || !edge_free(P, p, s.sc[e])) continue;
          long dd = dist2(q, old[W - 1][k]);
          if (best < 0 || dd < best_d || (dd == best_d && qi < best)) {
            best = qi;
            best_d = dd;
          }
        }
        reach[k] = at(P.g, best);
      }
    } else {
      for (int j = c + 1; j < W; ++j) {
        poses[j] = old[c];
        relax_out[2 * j] = -1;
      }
      for (int j = 0; j < W; ++j) write_pose(poses[j], poses_out + (size_t)j * 3 * (S + 1));
      *status_out = PATH_UNREACHABLE;
      return 0;
    }
  }
  std::vector<int> L(lens, lens + S);
  std::vector<V3> g = guide_points(L, reach, W);
  bool relaxed = false, broken = false;
  for (int j = c + 1; j < W; ++j) {
    int used = 0;
    Set T;
    if (j == W - 1) {
      T.assign(P.g.nvox(), 0);
      T[P.g.index(reach[S].x, reach[S].y, reach[S].z)] = 1;
    } else {
      T = waypoint_target(P, g[j], eps2, eps2_max, &used);
      if (used != eps2) relaxed = true;
    }
    std::vector<Set> V = waypoint_V(P, F, T);
    std::vector<V3> pose;
    int m = smooth_ladder(P, V, poses[j - 1], delta, max_relax, &pose);
    relax_out[2 * j + 1] = used;
    if (m < 0) {
      broken = true;
      poses[j] = poses[j - 1];
      relax_out[2 * j] = -1;
    } else {
      if (m > 0) relaxed = true;
      poses[j] = pose;
      relax_out[2 * j] = m;
    }
  }
  for (int j = 0; j < W; ++j) write_pose(poses[j], poses_out + (size_t)j * 3 * (S + 1));
  *status_out = broken ? PATH_BROKEN : (relaxed ? PATH_RELAXED : PATH_OK);
  return 0;
}

// Survivor sets of waypoints j_lo .. j_hi-1 only (same rules as
// orc_waypoint_sets); vsets_out [j_hi - j_lo][S+1][nvox].
int orc_waypoint_sets_range(int nx, int ny, int nz, const uint8_t* occ, int S, const int32_t* lens,
                            const int32_t* lo2, const int32_t* hi2, const int32_t* reach_pose, int W,
                            int j_lo, int j_hi, int eps2, int eps2_max, int32_t* eps2_used,
                            uint8_t* vsets_out) {
  Problem P = make_problem(nx, ny, nz, occ, S, lo2, hi2);
  std::vector<V3> reach = read_pose(reach_pose, S);
  std::vector<int> L(lens, lens + S);
  std::vector<V3> g = guide_points(L, reach, W);
  std::vector<Set> F = forward_sets(P, reach[0]);
  for (int j = j_lo; j < j_hi; ++j) {
    Set T;
    int used = 0;
    if (j == W - 1) {
      T.assign(P.g.nvox(), 0);
      T[P.g.index(reach[S].x, reach[S].y, reach[S].z)] = 1;
    } else {
      T = waypoint_target(P, g[j], eps2, eps2_max, &used);
    }
    eps2_used[j - j_lo] = used;
    std::vector<Set> V = waypoint_V(P, F, T);
    for (int k = 0; k <= S; ++k)
      std::memcpy(vsets_out + ((size_t)(j - j_lo) * (S + 1) + k) * P.g.nvox(), V[k].data(), P.g.nvox());
  }
  return 0;
}

// One smooth step with its relaxation ladder, given survivor sets V (bytes,
// [S+1][nvox]) and the reference pose.  Returns the number of increments
// used (written to *m_out, -1 when none fits) and the pose.
int orc_smooth_step(int nx, int ny, int nz, const uint8_t* occ, int S, const int32_t* lo2,
                    const int32_t* hi2, const uint8_t* vsets, const int32_t* ref_pose, int delta,
                    int max_relax, int32_t* pose_out, int32_t* m_out) {
  Problem P = make_problem(nx, ny, nz, occ, S, lo2, hi2);
  std::vector<Set> V(S + 1);
  for (int k = 0; k <= S; ++k)
    V[k].assign(vsets + (size_t)k * P.g.nvox(), vsets + (size_t)(k + 1) * P.g.nvox());
  std::vector<V3> pose;
  int m = smooth_ladder(P, V, read_pose(ref_pose, S), delta, max_relax, &pose);
  *m_out = m;
  if (m >= 0) write_pose(pose, pose_out);
  return 0;
}

// Algorithmic work of one propagation D_k(X) in bitset words: over every
// offset e of the shell and every 32-voxel word p (x-packed rows, Nx a
// multiple of 32) whose shifted input X[p+e] is non-zero, count the word and
// the supercover size of e.  Returns pairs; *sc_terms gets sum |SC(e)| over
// the counted pairs.
long orc_count_pairs(int nx, int ny, int nz, int lo2, int hi2, const uint8_t* X, long* sc_terms) {
  Grid g{nx, ny, nz};
  Segment s = make_segment(lo2, hi2);
  long pairs = 0, terms = 0;
  const int W = nx / 32;
  for (size_t e = 0; e < s.offs.size(); ++e) {
    const V3 d = s.offs[e];
    for (int z = 0; z < nz; ++z)
      for (int y = 0; y < ny; ++y)
        for (int w = 0; w < W; ++w) {
          bool nz_word = false;
          for (int b = 0; b < 32 && !nz_word; ++b) {
            int x = 32 * w + b;
            V3 q{x + d.x, y + d.y, z + d.z};
            if (g.inside(q.x, q.y, q.z) && X[g.index(q.x, q.y, q.z)]) nz_word = true;
          }
          if (nz_word) {
            ++pairs;
            terms += (long)s.sc[e].size();
          }
        }
  }
  *sc_terms = terms;
  return pairs;
}

}  // extern "C"
