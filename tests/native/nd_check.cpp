// Host check of the nested-dissection factorisation (nd_factor.cpp): for a
// seeded random operator with the library's stencil pattern (9 points, the
// pole rows reaching j = 2 and N - 3), solves A e = r with the host version of
// the GPU's two sweeps and prints the relative residual |r - A e| / |r| for
// the FP64 and the FP32 front matrices, and the factor's size.
//   nd_check M N leaf seed
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <random>
#include <string>
#include <vector>

#include "../../paper_2307_11107_gb300/csrc/nd_factor.h"

struct Op {
  int M, N;
  std::vector<double> c;  // [M][N][10]
  double get(int i, int j, int slot) const { return c[((size_t)(i - 1) * N + j) * 10 + slot]; }
};

static double coef(const void* ctx, int i, int j, int slot) { return ((const Op*)ctx)->get(i, j, slot); }

int main(int argc, char** argv) {
  if (argc < 5) return 2;
  Op op;
  op.M = std::atoi(argv[1]);
  op.N = std::atoi(argv[2]);
  const int leaf = std::atoi(argv[3]);
  std::mt19937_64 rng(std::strtoull(argv[4], nullptr, 10));
  std::uniform_real_distribution<double> U(-1.0, 1.0);
  const int M = op.M, N = op.N;
  op.c.assign((size_t)M * N * 10, 0.0);
  for (int i = 1; i <= M; ++i)
    for (int j = 0; j < N; ++j) {
      double* r = &op.c[((size_t)(i - 1) * N + j) * 10];
      double off = 0.0;
      // x1 coupling strong near the grain, x2 coupling strong far out (as Eq. 7's coefficients)
      const double a1 = std::pow(1.0 + 3.0 * (M - i) / M, 4.0), a2 = 1.0;
      for (int s = 0; s < 9; ++s) {
        if (s == 4) continue;
        const int di = s / 3 - 1, dj = s % 3 - 1;
        if ((j == 0 || j == N - 1) && dj != 0) continue;  // pole rows: no x2 neighbours but the reach below
        double v = (di && dj) ? 0.2 * U(rng) : (di ? a1 : a2) * (1.0 + 0.3 * U(rng));
        r[s] = v;
        off += std::fabs(v);
      }
      if (j == 0 || j == N - 1) {
        r[j == 0 ? 5 : 3] = 2.0 * (1.0 + 0.3 * U(rng));
        r[9] = -0.5 * (1.0 + 0.3 * U(rng));
        off += std::fabs(r[j == 0 ? 5 : 3]) + std::fabs(r[9]);
      }
      r[4] = -(1.05 + 0.2 * std::fabs(U(rng))) * off;
    }
  apic::NdFactor f;
  std::string why;
  if (!apic::nd_build(M, N, coef, &op, leaf, 4, true, f, why)) {
    std::printf("FAIL %s\n", why.c_str());
    return 1;
  }
  std::vector<double> r((size_t)M * N), e((size_t)M * N);
  for (double& x : r) x = U(rng);
  double worst[2];
  for (int prec = 0; prec < 2; ++prec) {
    apic::nd_solve_host(f, r.data(), e.data(), prec == 0);
    double num = 0.0, den = 0.0;
    for (int i = 1; i <= M; ++i)
      for (int j = 0; j < N; ++j) {
        double ae = 0.0;
        for (int s = 0; s < 10; ++s) {
          int di, dj;
          if (s < 9) {
            di = s / 3 - 1;
            dj = s % 3 - 1;
          } else {
            di = 0;
            if (j == 0) dj = 2;
            else if (j == N - 1) dj = -2;
            else continue;
          }
          const int a = i + di, b = j + dj;
          if (a < 1 || a > M || b < 0 || b >= N) continue;
          ae += op.get(i, j, s) * e[(size_t)(a - 1) * N + b];
        }
        const double d = r[(size_t)(i - 1) * N + j] - ae;
        num += d * d;
        den += r[(size_t)(i - 1) * N + j] * r[(size_t)(i - 1) * N + j];
      }
    worst[prec] = std::sqrt(num / den);
  }
  // the device tables: a first instance (the same factor) shifts every
  // global offset of the second; the table sweeps of the second must equal
  // the host sweeps with the FP32 matrices
  apic::NdUpload up;
  apic::NdLevels l0, l1;
  const int64_t mat1 = ((f.fm_total + f.nb_total + 63) / 64) * 64, w1 = ((f.w_total + 63) / 64) * 64;
  apic::nd_layout(f, 0, 0, 64, 192, 2048, 16384, 2048, 8, 16384, 304, up, l0);
  apic::nd_layout(f, mat1, w1, 64, 192, 2048, 16384, 2048, 8, 16384, 304, up, l1);
  std::vector<float> matbuf((size_t)(2 * mat1), 0.0f);
  for (int k = 0; k < 2; ++k) {
    std::copy(f.fm.begin(), f.fm.end(), matbuf.begin() + k * mat1);
    std::copy(f.nb.begin(), f.nb.end(), matbuf.begin() + k * mat1 + f.fm_total);
  }
  // every task's matrix rows are one contiguous range in each sweep (the
  // device stages a task by one copy): consecutive fronts of a task follow
  // one another
  long long gaps = 0, big = 0;
  for (size_t i = 0; i < up.tasks.size(); ++i) {
    const apic::NdTask& t = up.tasks[i];
    const bool fwd = (int)i < l0.bt[0] || ((int)i >= l1.ft[0] && (int)i < l1.bt[0]);
    int64_t fw = 0, bw = 0;
    for (int q = t.front; t.warp != 0 && q < t.front + t.n; ++q) {
      const apic::NdFront &A = up.fronts[q];
      fw += (int64_t)(A.s + A.u) * A.sp;
      bw += (int64_t)A.s * A.up;
      if (q + 1 == t.front + t.n) break;
      const apic::NdFront &C = up.fronts[q + 1];
      gaps += A.FM + (int64_t)(A.s + A.u) * A.sp != C.FM;
      gaps += A.NB + (int64_t)A.s * A.up != C.NB;
    }
    if (t.warp == 0) {
      const apic::NdFront &A = up.fronts[t.front];
      fw = (int64_t)t.n * A.sp;
      bw = (int64_t)t.n * A.up;
    }
    big += (fwd ? fw : bw) > 16384;  // the task's matrix rows fit a worker's stage
  }
  if (gaps || big) {
    std::printf("FAIL %lld task fronts not contiguous, %lld tasks beyond the stage\n", gaps, big);
    return 1;
  }
  std::vector<float> r32(r.begin(), r.end()), e32((size_t)M * N, 0.0f), w((size_t)(2 * w1), 0.0f);
  apic::nd_solve_tables(up, l1, f.depth, matbuf, N, r32.data(), e32.data(), w);
  std::vector<double> eh((size_t)M * N);
  apic::nd_solve_host(f, r.data(), eh.data(), false);
  double dmax = 0.0, emax = 0.0;
  for (size_t q = 0; q < eh.size(); ++q) {
    dmax = std::max(dmax, std::fabs((double)e32[q] - eh[q]));
    emax = std::max(emax, std::fabs(eh[q]));
  }
  std::printf("OK %.3e %.3e fronts %zu depth %d floats %lld tables %.3e\n", worst[0], worst[1], f.fronts.size(),
              f.depth, (long long)(f.fm_total + f.nb_total), dmax / emax);
  return 0;
}
