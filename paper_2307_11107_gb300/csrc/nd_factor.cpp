// Nested-dissection factorisation of the Poisson correction system (see
// nd_factor.h).  Host-only C++: ordering, symbolic fronts, multifrontal LU in
// FP64 (dense fronts, children's Schur complements added into their
// parent), and the host version of the GPU's two sweeps.
#include "nd_factor.h"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <thread>

namespace apic {
namespace {

struct Rect {
  int i0, i1, j0, j1;  // unknown rows [i0, i1) (0-based: grid row i0 + 1), columns [j0, j1)
  long long area() const { return (long long)(i1 - i0) * (j1 - j0); }
  bool empty() const { return i1 <= i0 || j1 <= j0; }
};

struct Builder {
  int M, N, leaf;
  NdFactor& f;
  std::vector<Rect> rect;         // the subtree rectangle of every front
  std::vector<std::vector<int32_t>> sep, upd;
  Builder(int M_, int N_, int leaf_, NdFactor& f_) : M(M_), N(N_), leaf(leaf_), f(f_) {}

  int add_front(const Rect& r, std::vector<int32_t>&& s, int c0, int c1, int level) {
    NdFront fr;
    std::memset(&fr, 0, sizeof(fr));
    fr.level = level;
    fr.child[0] = c0;
    fr.child[1] = c1;
    fr.parent = -1;
    int id = (int)f.fronts.size();
    if (c0 >= 0) f.fronts[c0].parent = id;
    if (c1 >= 0) f.fronts[c1].parent = id;
    f.fronts.push_back(fr);
    rect.push_back(r);
    sep.push_back(std::move(s));
    return id;
  }

  // Children before their parent (post-order).
  int build(const Rect& r, int level) {
    const int h = r.i1 - r.i0, w = r.j1 - r.j0;
    auto leaf_front = [&]() {
      std::vector<int32_t> s;
      for (int i = r.i0; i < r.i1; ++i)
        for (int j = r.j0; j < r.j1; ++j) s.push_back(i * N + j);
      return add_front(r, std::move(s), -1, -1, level);
    };
    if (r.area() <= leaf || (h < 3 && w < 3)) return leaf_front();
    if (h >= w && h >= 3) {
      const int im = r.i0 + (h - 1) / 2;
      Rect a{r.i0, im, r.j0, r.j1}, b{im + 1, r.i1, r.j0, r.j1};
      int c0 = a.empty() ? -1 : build(a, level + 1);
      int c1 = b.empty() ? -1 : build(b, level + 1);
      std::vector<int32_t> s;
      for (int j = r.j0; j < r.j1; ++j) s.push_back(im * N + j);
      return add_front(r, std::move(s), c0, c1, level);
    }
    // column cut, never at j = 1 or N - 2 (jumped by the pole couplings)
    int jm = r.j0 + (w - 1) / 2;
    if (jm == 1) jm = 2;
    if (jm == N - 2) jm = N - 3;
    if (jm <= r.j0 || jm >= r.j1 - 1) {
      if (h >= 3) {  // cut the rows instead
        const int im = r.i0 + (h - 1) / 2;
        Rect a{r.i0, im, r.j0, r.j1}, b{im + 1, r.i1, r.j0, r.j1};
        int c0 = a.empty() ? -1 : build(a, level + 1);
        int c1 = b.empty() ? -1 : build(b, level + 1);
        std::vector<int32_t> s;
        for (int j = r.j0; j < r.j1; ++j) s.push_back(im * N + j);
        return add_front(r, std::move(s), c0, c1, level);
      }
      return leaf_front();
    }
    Rect a{r.i0, r.i1, r.j0, jm}, b{r.i0, r.i1, jm + 1, r.j1};
    int c0 = a.empty() ? -1 : build(a, level + 1);
    int c1 = b.empty() ? -1 : build(b, level + 1);
    std::vector<int32_t> s;
    for (int i = r.i0; i < r.i1; ++i) s.push_back(i * N + jm);
    return add_front(r, std::move(s), c0, c1, level);
  }

  // Structural neighbours of node (i, j), symmetric (row and column couplings).
  template <class Fn>
  void neighbours(int i, int j, Fn fn) const {
    for (int di = -1; di <= 1; ++di)
      for (int dj = -1; dj <= 1; ++dj) {
        if (!di && !dj) continue;
        int a = i + di, b = j + dj;
        if (a >= 0 && a < M && b >= 0 && b < N) fn(a * N + b);
      }
    if (j == 0) fn(i * N + 2);
    if (j == 2) fn(i * N + 0);
    if (j == N - 1) fn(i * N + N - 3);
    if (j == N - 3) fn(i * N + N - 1);
  }

  // U = nodes outside the rectangle coupled to a node inside (only nodes
  // within two columns or one row of its border can have such neighbours).
  std::vector<int32_t> update_set(const Rect& r) const {
    std::vector<int32_t> u;
    auto inside = [&](int n) {
      int i = n / N, j = n % N;
      return i >= r.i0 && i < r.i1 && j >= r.j0 && j < r.j1;
    };
    for (int i = r.i0; i < r.i1; ++i)
      for (int j = r.j0; j < r.j1; ++j) {
        if (i > r.i0 && i < r.i1 - 1 && j > r.j0 + 1 && j < r.j1 - 2) continue;
        neighbours(i, j, [&](int n) {
          if (!inside(n)) u.push_back(n);
        });
      }
    std::sort(u.begin(), u.end());
    u.erase(std::unique(u.begin(), u.end()), u.end());
    return u;
  }
};

// C[m x n] (ldc) -= A[m x k] (lda) B[k x n] (ldb), rows of C split over `threads`.
void gemm_sub(int m, int n, int k, const double* A, int lda, const double* B, int ldb, double* C, int ldc,
              int threads) {
  auto rows = [&](int r0, int r1) {
    for (int i = r0; i < r1; ++i) {
      double* c = C + (size_t)i * ldc;
      const double* a = A + (size_t)i * lda;
      for (int p = 0; p < k; ++p) {
        const double ap = a[p];
        if (ap == 0.0) continue;
        const double* b = B + (size_t)p * ldb;
        for (int j = 0; j < n; ++j) c[j] -= ap * b[j];
      }
    }
  };
  if (threads <= 1 || (long long)m * n * k < 4000000) {
    rows(0, m);
    return;
  }
  std::vector<std::thread> th;
  int per = (m + threads - 1) / threads;
  for (int t = 0; t < threads; ++t) {
    int r0 = t * per, r1 = std::min(m, r0 + per);
    if (r0 >= r1) break;
    th.emplace_back(rows, r0, r1);
  }
  for (auto& t : th) t.join();
}

// In-place inverse of the n x n row-major matrix a (Gauss-Jordan, partial
// pivoting).  Returns false if a pivot vanishes.
bool invert(double* a, int n, int threads) {
  std::vector<int> perm(n);
  for (int i = 0; i < n; ++i) perm[i] = i;
  std::vector<double> inv((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) inv[(size_t)i * n + i] = 1.0;
  for (int c = 0; c < n; ++c) {
    int p = c;
    double best = std::fabs(a[(size_t)c * n + c]);
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(a[(size_t)r * n + c]) > best) {
        best = std::fabs(a[(size_t)r * n + c]);
        p = r;
      }
    if (!(best > 0.0) || !std::isfinite(best)) return false;
    if (p != c) {
      for (int j = 0; j < n; ++j) {
        std::swap(a[(size_t)p * n + j], a[(size_t)c * n + j]);
        std::swap(inv[(size_t)p * n + j], inv[(size_t)c * n + j]);
      }
    }
    const double d = 1.0 / a[(size_t)c * n + c];
    for (int j = 0; j < n; ++j) {
      a[(size_t)c * n + j] *= d;
      inv[(size_t)c * n + j] *= d;
    }
    auto elim = [&](int r0, int r1) {
      for (int r = r0; r < r1; ++r) {
        if (r == c) continue;
        const double m = a[(size_t)r * n + c];
        if (m == 0.0) continue;
        double* ar = a + (size_t)r * n;
        double* ir = inv.data() + (size_t)r * n;
        const double* ac = a + (size_t)c * n;
        const double* ic = inv.data() + (size_t)c * n;
        for (int j = 0; j < n; ++j) {
          ar[j] -= m * ac[j];
          ir[j] -= m * ic[j];
        }
      }
    };
    if (threads > 1 && n >= 384) {
      std::vector<std::thread> th;
      int per = (n + threads - 1) / threads;
      for (int t = 0; t < threads; ++t) {
        int r0 = t * per, r1 = std::min(n, r0 + per);
        if (r0 >= r1) break;
        th.emplace_back(elim, r0, r1);
      }
      for (auto& t : th) t.join();
    } else {
      elim(0, n);
    }
  }
  std::memcpy(a, inv.data(), sizeof(double) * (size_t)n * n);
  return true;
}

}  // namespace

bool nd_build(int M, int N, NdCoef coef, const void* ctx, int leaf, int threads, bool keep64, NdFactor& f,
              std::string& why) {
  f = NdFactor();
  f.M = M;
  f.N = N;
  if (M < 1 || N < 5) {
    why = "grid too small for the nested dissection";
    return false;
  }
  threads = std::max(1, threads);
  Builder b(M, N, std::max(1, leaf), f);
  b.build(Rect{0, M, 0, N}, 0);
  const int nf = (int)f.fronts.size();
  // separators own every unknown exactly once
  std::vector<int32_t> owner((size_t)M * N, -1);
  for (int k = 0; k < nf; ++k)
    for (int32_t n : b.sep[k]) {
      if (owner[n] >= 0) {
        why = "node in two separators";
        return false;
      }
      owner[n] = k;
    }
  for (size_t n = 0; n < owner.size(); ++n)
    if (owner[n] < 0) {
      why = "node in no separator";
      return false;
    }
  // update sets, checked to lie on ancestors' separators
  b.upd.resize(nf);
  for (int k = 0; k < nf; ++k) {
    b.upd[k] = b.update_set(b.rect[k]);
    for (int32_t n : b.upd[k]) {
      int a = f.fronts[k].parent;
      while (a >= 0 && a != owner[n]) a = f.fronts[a].parent;
      if (a < 0) {
        why = "update set outside the ancestors' separators";
        return false;
      }
    }
  }
  // layout
  int64_t w = 0, fm = 0, nb = 0, g = 0, ix = 0;
  for (int k = 0; k < nf; ++k) {
    NdFront& F = f.fronts[k];
    F.s = (int)b.sep[k].size();
    F.u = (int)b.upd[k].size();
    F.sp = (F.s + 3) & ~3;
    F.up = (F.u + 3) & ~3;
    F.S = ix;
    ix += F.s;
    F.U = ix;
    ix += F.u;
    F.G = g;
    g += 2 * (int64_t)(F.s + F.u);
    F.W = w;
    w += (F.u + 3) & ~3;
    f.depth = std::max(f.depth, F.level);
    f.max_s = std::max(f.max_s, F.s);
    f.max_u = std::max(f.max_u, F.u);
  }
  // matrices level by level, deepest first (the order of the device's task
  // tables: a task's fronts hold one contiguous range, staged by one copy)
  for (int l = f.depth; l >= 0; --l)
    for (int k = 0; k < nf; ++k) {
      NdFront& F = f.fronts[k];
      if (F.level != l) continue;
      F.FM = fm;
      fm += (int64_t)(F.s + F.u) * F.sp;
      F.NB = nb;
      nb += (int64_t)F.s * F.up;
    }
  f.w_total = w;
  f.fm_total = fm;
  f.nb_total = nb;
  f.idx.resize((size_t)ix);
  f.gather.assign((size_t)g, -1);
  f.by_level.assign(f.depth + 1, {});
  for (int k = 0; k < nf; ++k) {
    const NdFront& F = f.fronts[k];
    std::copy(b.sep[k].begin(), b.sep[k].end(), f.idx.begin() + F.S);
    std::copy(b.upd[k].begin(), b.upd[k].end(), f.idx.begin() + F.U);
    f.by_level[F.level].push_back(k);
  }
  // gather tables: where each child's update vector lands in [S; U]
  {
    std::vector<int32_t> pos((size_t)M * N, -1);
    for (int k = 0; k < nf; ++k) {
      const NdFront& F = f.fronts[k];
      for (int a = 0; a < F.s + F.u; ++a) pos[f.idx[F.S + a]] = a;  // S and U are adjacent in idx
      for (int c = 0; c < 2; ++c) {
        if (F.child[c] < 0) continue;
        const NdFront& C = f.fronts[F.child[c]];
        for (int q = 0; q < C.u; ++q) {
          int p = pos[f.idx[C.U + q]];
          if (p < 0) {
            why = "child update set not inside its parent's front";
            return false;
          }
          f.gather[F.G + 2 * p + c] = q;
        }
      }
      for (int a = 0; a < F.s + F.u; ++a) pos[f.idx[F.S + a]] = -1;
    }
  }
  // numeric factorisation, deepest level first; the fronts of one level are
  // independent
  f.fm.assign((size_t)fm, 0.0f);
  f.nb.assign((size_t)nb, 0.0f);
  if (keep64) {
    f.fm64.assign((size_t)fm, 0.0);
    f.nb64.assign((size_t)nb, 0.0);
  }
  std::vector<std::vector<double>> updm(nf);
  std::atomic<int> bad(0);
  auto factor_front = [&](int k, int inner_threads, std::vector<int32_t>& pos) {
    const NdFront& F = f.fronts[k];
    const int s = F.s, u = F.u, n = s + u;
    const int32_t* SU = f.idx.data() + F.S;
    for (int a = 0; a < n; ++a) pos[SU[a]] = a;
    std::vector<double> A((size_t)n * n, 0.0);
    // original couplings: rows of S with columns in S or U; rows of U with columns in S
    auto row_entries = [&](int node, int row_pos, bool only_S_cols) {
      const int i = node / N, j = node % N;  // unknown row i <-> grid row i + 1
      for (int slot = 0; slot < 10; ++slot) {
        int di, dj;
        if (slot < 9) {
          di = slot / 3 - 1;
          dj = slot % 3 - 1;
        } else {
          di = 0;
          if (j == 0) dj = 2;
          else if (j == N - 1) dj = -2;
          else continue;
        }
        const int a = i + di, c = j + dj;
        if (a < 0 || a >= M || c < 0 || c >= N) continue;
        const int p = pos[a * N + c];
        if (p < 0 || (only_S_cols && p >= s)) continue;
        const double v = coef(ctx, i + 1, j, slot);
        if (v != 0.0) A[(size_t)row_pos * n + p] += v;
      }
    };
    for (int a = 0; a < s; ++a) row_entries(SU[a], a, false);
    for (int q = 0; q < u; ++q) row_entries(SU[s + q], s + q, true);
    // children's Schur complements
    for (int c = 0; c < 2; ++c) {
      if (F.child[c] < 0) continue;
      const NdFront& C = f.fronts[F.child[c]];
      std::vector<int> map(C.u);
      for (int q = 0; q < C.u; ++q) map[q] = pos[f.idx[C.U + q]];
      const std::vector<double>& Uc = updm[F.child[c]];
      for (int q = 0; q < C.u; ++q) {
        double* row = A.data() + (size_t)map[q] * n;
        const double* src = Uc.data() + (size_t)q * C.u;
        for (int t = 0; t < C.u; ++t) row[map[t]] += src[t];
      }
      std::vector<double>().swap(updm[F.child[c]]);
    }
    for (int a = 0; a < n; ++a) pos[SU[a]] = -1;
    // F_SS^-1
    std::vector<double> Fi((size_t)s * s);
    for (int a = 0; a < s; ++a) std::memcpy(Fi.data() + (size_t)a * s, A.data() + (size_t)a * n, sizeof(double) * s);
    if (!invert(Fi.data(), s, inner_threads)) {
      bad = 1;
      return;
    }
    // Mp = F_US F_SS^-1 (u x s), Nb = F_SS^-1 F_SU (s x u), Upd = F_UU - Mp F_SU
    std::vector<double> Mp((size_t)u * s, 0.0), Nb((size_t)s * u, 0.0);
    if (u > 0) {
      // computed as 0 - (-A) B with gemm_sub
      std::vector<double> negUS((size_t)u * s), negSS((size_t)s * s);
      for (int q = 0; q < u; ++q)
        for (int a = 0; a < s; ++a) negUS[(size_t)q * s + a] = -A[(size_t)(s + q) * n + a];
      gemm_sub(u, s, s, negUS.data(), s, Fi.data(), s, Mp.data(), s, inner_threads);
      std::vector<double> SUm((size_t)s * u);
      for (int a = 0; a < s; ++a)
        for (int q = 0; q < u; ++q) SUm[(size_t)a * u + q] = A[(size_t)a * n + s + q];
      for (size_t z = 0; z < negSS.size(); ++z) negSS[z] = -Fi[z];
      gemm_sub(s, u, s, negSS.data(), s, SUm.data(), u, Nb.data(), u, inner_threads);
      std::vector<double> Up((size_t)u * u);
      for (int q = 0; q < u; ++q)
        for (int t = 0; t < u; ++t) Up[(size_t)q * u + t] = A[(size_t)(s + q) * n + s + t];
      gemm_sub(u, u, s, Mp.data(), s, SUm.data(), u, Up.data(), u, inner_threads);
      updm[k] = std::move(Up);
    }
    // store: FM rows 0..s-1 = F_SS^-1, rows s..s+u-1 = Mp; NB = Nb
    for (int a = 0; a < s; ++a)
      for (int t = 0; t < s; ++t) {
        const double v = Fi[(size_t)a * s + t];
        f.fm[F.FM + (size_t)a * F.sp + t] = (float)v;
        if (keep64) f.fm64[F.FM + (size_t)a * F.sp + t] = v;
      }
    for (int q = 0; q < u; ++q)
      for (int t = 0; t < s; ++t) {
        const double v = Mp[(size_t)q * s + t];
        f.fm[F.FM + (size_t)(s + q) * F.sp + t] = (float)v;
        if (keep64) f.fm64[F.FM + (size_t)(s + q) * F.sp + t] = v;
      }
    for (int a = 0; a < s; ++a)
      for (int q = 0; q < u; ++q) {
        const double v = Nb[(size_t)a * u + q];
        f.nb[F.NB + (size_t)a * F.up + q] = (float)v;
        if (keep64) f.nb64[F.NB + (size_t)a * F.up + q] = v;
      }
  };
  for (int lv = f.depth; lv >= 0 && !bad; --lv) {
    const std::vector<int>& L = f.by_level[lv];
    if ((int)L.size() >= threads && threads > 1) {
      std::atomic<int> next(0);
      std::vector<std::thread> th;
      for (int t = 0; t < threads; ++t)
        th.emplace_back([&]() {
          std::vector<int32_t> pos((size_t)M * N, -1);
          for (int q = next++; q < (int)L.size() && !bad; q = next++) factor_front(L[q], 1, pos);
        });
      for (auto& t : th) t.join();
    } else {
      std::vector<int32_t> pos((size_t)M * N, -1);
      for (int k : L) {
        factor_front(k, threads, pos);
        if (bad) break;
      }
    }
  }
  if (bad) {
    why = "singular front in the nested-dissection factorisation";
    return false;
  }
  return true;
}

void nd_solve_host(const NdFactor& f, const double* r, double* e, bool fp64) {
  const bool d = fp64 && !f.fm64.empty();
  auto FM = [&](int64_t o) { return d ? f.fm64[o] : (double)f.fm[o]; };
  auto NB = [&](int64_t o) { return d ? f.nb64[o] : (double)f.nb[o]; };
  std::vector<double> w((size_t)f.w_total, 0.0), v;
  for (int lv = f.depth; lv >= 0; --lv)
    for (int k : f.by_level[lv]) {
      const NdFront& F = f.fronts[k];
      const int s = F.s, u = F.u;
      v.assign(s + u, 0.0);
      for (int p = 0; p < s + u; ++p) {
        double x = p < s ? r[f.idx[F.S + p]] : 0.0;
        for (int c = 0; c < 2; ++c) {
          const int q = f.gather[F.G + 2 * p + c];
          if (q >= 0) x += w[f.fronts[F.child[c]].W + q];
        }
        v[p] = x;
      }
      for (int a = 0; a < s + u; ++a) {
        double acc = 0.0;
        for (int t = 0; t < s; ++t) acc += FM(F.FM + (int64_t)a * F.sp + t) * v[t];
        if (a < s) e[f.idx[F.S + a]] = acc;
        else w[F.W + (a - s)] = v[a] - acc;
      }
    }
  for (int lv = 0; lv <= f.depth; ++lv)
    for (int k : f.by_level[lv]) {
      const NdFront& F = f.fronts[k];
      for (int a = 0; a < F.s; ++a) {
        double acc = 0.0;
        for (int q = 0; q < F.u; ++q) acc += NB(F.NB + (int64_t)a * F.up + q) * e[f.idx[F.U + q]];
        e[f.idx[F.S + a]] -= acc;
      }
    }
}

int nd_layout(const NdFactor& f, int64_t mat, int64_t wb, int warp_s, int warp_u, int warp_floats, int task_floats,
              int task_rows, int task_fronts, int stage_floats, int ctas, NdUpload& up, NdLevels& lv) {
  const int nf = (int)f.fronts.size();
  const int64_t front0 = (int64_t)up.fronts.size(), idx0 = (int64_t)up.idx.size(), g0 = (int64_t)up.gather.size();
  std::vector<int> order;  // deepest level first
  for (int l = f.depth; l >= 0; --l)
    for (int k : f.by_level[l]) order.push_back(k);
  std::vector<int> where(nf);
  for (int q = 0; q < nf; ++q) where[order[q]] = q;
  // large in a sweep: beyond a warp's vector areas, or a matrix beyond what a
  // warp stages in shared memory
  auto large_in = [&](const NdFront& F, bool fwd) {
    const int64_t floats = fwd ? (int64_t)(F.s + F.u) * F.sp : (int64_t)F.s * F.up;
    return F.s > warp_s || F.u > warp_u || floats > warp_floats;
  };
  auto large = [&](const NdFront& F) { return large_in(F, true) || large_in(F, false); };
  int need = 0;
  for (int q = 0; q < nf; ++q) {
    NdFront F = f.fronts[order[q]];
    for (int c = 0; c < 2; ++c)
      if (F.child[c] >= 0) F.child[c] = (int)(front0 + where[F.child[c]]);
    if (F.parent >= 0) F.parent = (int)(front0 + where[F.parent]);
    F.S += idx0;
    F.U += idx0;
    F.G += g0;
    F.W += wb;
    F.FM += mat;
    F.NB += mat + f.fm_total;
    if (large(F)) need = std::max(need, std::max(F.sp, F.up));
    up.fronts.push_back(F);
  }
  up.idx.insert(up.idx.end(), f.idx.begin(), f.idx.end());
  up.gather.insert(up.gather.end(), f.gather.begin(), f.gather.end());
  for (int q = 0; q < nf; ++q) {  // child-relative gather entries -> absolute update-vector offsets
    const NdFront& F = up.fronts[front0 + q];
    for (int p = 0; p < F.s + F.u; ++p)
      for (int c = 0; c < 2; ++c) {
        int32_t& g = up.gather[F.G + 2 * p + c];
        if (g >= 0) g = (int32_t)(up.fronts[F.child[c]].W + g);
      }
  }
  // tiny fronts (s <= 16, u <= 48) go four to a warp, one per 8-lane group
  // every task's matrix rows fit the device's staging buffer (stage_floats)
  auto floats_in = [&](const NdFront& F, bool fwd) {
    return fwd ? (int64_t)(F.s + F.u) * F.sp : (int64_t)F.s * F.up;
  };
  auto level_tasks = [&](int l, bool fwd) {
    auto large = [&](const NdFront& F) { return large_in(F, fwd); };
    auto tiny0 = [&](const NdFront& F) { return F.s <= kNdTinyS && F.u <= kNdTinyU && !large(F); };
    int q = 0;
    while (q < nf && up.fronts[front0 + q].level != l) ++q;
    int small = 0, nt = 0;
    for (int z = q; z < nf && up.fronts[front0 + z].level == l; ++z) {
      small += !large(up.fronts[front0 + z]);
      nt += tiny0(up.fronts[front0 + z]);
    }
    const int c = std::max(1, ctas);
    // tiny fronts go four to a warp when there are at least four per CTA,
    // else one to a warp like the small ones
    const bool use_tiny = nt >= 4 * c;
    auto tiny = [&](const NdFront& F) { return use_tiny && tiny0(F); };
    const int per = std::max(1, std::min(task_fronts, (small + c - 1) / c));
    const int per_tiny = std::max(1, std::min(4 * task_fronts, (nt + c - 1) / c));
    while (q < nf && up.fronts[front0 + q].level == l) {
      const NdFront& F = up.fronts[front0 + q];
      if (large(F)) {
        const int rows = fwd ? F.s + F.u : F.s;
        const int width = fwd ? F.sp : std::max(4, F.up);
        const int nr = std::max(1, std::min(task_rows, task_floats / width));
        for (int r = 0; r < rows; r += nr) up.tasks.push_back(NdTask{(int)(front0 + q), r, std::min(nr, rows - r), 0});
        ++q;
        continue;
      }
      const bool t = tiny(F);
      const int cap = t ? per_tiny : per;
      int n = 0;
      int64_t floats = 0;
      while (q + n < nf && n < cap) {
        const NdFront& G = up.fronts[front0 + q + n];
        if (G.level != l || large(G) || tiny(G) != t || floats + floats_in(G, fwd) > stage_floats) break;
        floats += floats_in(G, fwd);
        ++n;
      }
      up.tasks.push_back(NdTask{(int)(front0 + q), 0, n, t ? 2 : 1});
      q += n;
    }
  };
  lv.ft.assign(f.depth + 2, 0);
  lv.bt.assign(f.depth + 2, 0);
  for (int l = 0; l <= f.depth; ++l) {
    lv.ft[l] = (int32_t)up.tasks.size();
    level_tasks(l, true);
  }
  lv.ft[f.depth + 1] = (int32_t)up.tasks.size();
  for (int l = 0; l <= f.depth; ++l) {
    lv.bt[l] = (int32_t)up.tasks.size();
    level_tasks(l, false);
  }
  lv.bt[f.depth + 1] = (int32_t)up.tasks.size();
  return need;
}

void nd_solve_tables(const NdUpload& up, const NdLevels& lv, int depth, const std::vector<float>& matbuf, int N,
                     const float* r, float* e, std::vector<float>& w) {
  (void)N;
  auto rhs = [&](const NdFront& F, int p) {
    float v = p < F.s ? r[up.idx[F.S + p]] : 0.0f;
    const int g0 = up.gather[F.G + 2 * p], g1 = up.gather[F.G + 2 * p + 1];
    if (g0 >= 0) v += w[g0];
    if (g1 >= 0) v += w[g1];
    return v;
  };
  auto fwd = [&](const NdFront& F, int r0, int r1) {
    std::vector<float> v(F.sp, 0.0f);
    for (int p = 0; p < F.s; ++p) v[p] = rhs(F, p);
    for (int a = r0; a < r1; ++a) {
      float acc = 0.0f;
      for (int t = 0; t < F.sp; ++t) acc += matbuf[F.FM + (int64_t)a * F.sp + t] * v[t];
      if (a < F.s) e[up.idx[F.S + a]] = acc;
      else w[F.W + a - F.s] = rhs(F, a) - acc;
    }
  };
  auto back = [&](const NdFront& F, int r0, int r1) {
    std::vector<float> xu(std::max(F.up, 1), 0.0f);
    for (int q = 0; q < F.u; ++q) xu[q] = e[up.idx[F.U + q]];
    for (int a = r0; a < r1; ++a) {
      float acc = 0.0f;
      for (int q = 0; q < F.up; ++q) acc += matbuf[F.NB + (int64_t)a * F.up + q] * xu[q];
      e[up.idx[F.S + a]] -= acc;
    }
  };
  for (int l = depth; l >= 0; --l)
    for (int t = lv.ft[l]; t < lv.ft[l + 1]; ++t) {
      const NdTask& T = up.tasks[t];
      if (T.warp == 0) fwd(up.fronts[T.front], T.r0, T.r0 + T.n);
      else
        for (int k = 0; k < T.n; ++k) fwd(up.fronts[T.front + k], 0, up.fronts[T.front + k].s + up.fronts[T.front + k].u);
    }
  for (int l = 0; l <= depth; ++l)
    for (int t = lv.bt[l]; t < lv.bt[l + 1]; ++t) {
      const NdTask& T = up.tasks[t];
      if (T.warp == 0) back(up.fronts[T.front], T.r0, T.r0 + T.n);
      else
        for (int k = 0; k < T.n; ++k) back(up.fronts[T.front + k], 0, up.fronts[T.front + k].s);
    }
}

}  // namespace apic
