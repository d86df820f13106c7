// Host side of libapic: the C ABI of include/apic.h.  Set-up of the grid,
// node volumes (Eq. 5), sampling tables (Eqs. 4-5), the finite-difference
// operator of Eq. 7 and its Galerkin multigrid hierarchy; device memory; the
// per-step launch sequence, captured once into a CUDA graph whose BiCGSTAB loop
// is a device-controlled while-node.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "apic_internal.h"
#include "dual.cuh"
#include "geom.cuh"

using namespace apic;

namespace {

// ---- quadrature (Gauss-Legendre, 10 points, by Newton on the three-term recurrence) ----
struct GL10 {
  double x[10], w[10];
  GL10() {
    const int n = 10;
    for (int k = 0; k < n; ++k) {
      double z = std::cos(kPi * (k + 0.75) / (n + 0.5)), dp = 1.0;
      for (int it = 0; it < 200; ++it) {
        double pm = 1.0, p = z;
        for (int l = 2; l <= n; ++l) {
          double pn = ((2 * l - 1) * z * p - (l - 1) * pm) / l;
          pm = p;
          p = pn;
        }
        dp = n * (pm - z * p) / (1.0 - z * z);
        double step = p / dp;
        z -= step;
        if (std::fabs(step) < 1e-17) break;
      }
      x[k] = z;
      w[k] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
  }
};
const GL10& gl10() {
  static GL10 g;
  return g;
}

int bits_for(long long v) {
  int b = 0;
  while (v > 0) {
    ++b;
    v >>= 1;
  }
  return b;
}

double x1_node_h(const Inst& I, int i) { return i == I.n1 ? I.x1_out : -1.0 + i * I.h1; }
double x2_node_h(const Inst& I, int j) { return j == I.n2 ? 1.0 : -1.0 + j * I.h2; }

// Host stencil of one level: kSt arrays of nodes.
struct HostLevel {
  int n1, n2, N1, N2;
  std::vector<double> st;  // [kSt][nodes]
  long long nodes() const { return (long long)N1 * N2; }
  double& at(int k, int i, int j) { return st[(size_t)k * nodes() + (size_t)i * N2 + j]; }
  double get(int k, int i, int j) const { return st[(size_t)k * nodes() + (size_t)i * N2 + j]; }
};

// Galerkin coarse operator R A P with bilinear P (zero on Dirichlet rows) and
// R = P^T / 4; the result is a 3x3 stencil on every coarse row.
bool galerkin(const HostLevel& F, HostLevel& C, bool fine_pole) {
  C.n1 = F.n1 / 2;
  C.n2 = F.n2 / 2;
  C.N1 = C.n1 + 1;
  C.N2 = C.n2 + 1;
  C.st.assign((size_t)kSt * C.nodes(), 0.0);
  auto w = [](int d) { return d == 0 ? 1.0 : 0.5; };
  for (int I = 1; I < C.n1; ++I)
    for (int J = 0; J <= C.n2; ++J) {
      for (int di = -1; di <= 1; ++di) {
        int i = 2 * I + di;
        if (i < 1 || i > F.n1 - 1) continue;
        for (int dj = -1; dj <= 1; ++dj) {
          int j = 2 * J + dj;
          if (j < 0 || j > F.n2) continue;
          double wr = 0.25 * w(di) * w(dj);
          // fine row (i, j): its entries (i2, j2, s)
          struct E {
            int i2, j2;
            double s;
          } ent[11];
          int ne = 0;
          for (int a = -1; a <= 1; ++a)
            for (int b = -1; b <= 1; ++b) {
              int j2 = j + b;
              if (j2 < 0 || j2 > F.n2) continue;
              double s = F.get(st_slot(a, b), i, j);
              if (s != 0.0) ent[ne++] = {i + a, j2, s};
            }
          if (fine_pole) {
            double s = F.get(kStPole, i, j);
            if (s != 0.0) {
              if (j == 0) ent[ne++] = {i, 2, s};
              else if (j == F.n2) ent[ne++] = {i, F.n2 - 2, s};
            }
          }
          for (int e = 0; e < ne; ++e) {
            int i2 = ent[e].i2, j2 = ent[e].j2;
            int Ia = i2 / 2, Ib = (i2 + 1) / 2, Ja = j2 / 2, Jb = (j2 + 1) / 2;
            int Is[2] = {Ia, Ib}, Js[2] = {Ja, Jb};
            double wi = (i2 % 2 == 0) ? 1.0 : 0.5, wj = (j2 % 2 == 0) ? 1.0 : 0.5;
            int ni = (i2 % 2 == 0) ? 1 : 2, nj = (j2 % 2 == 0) ? 1 : 2;
            for (int u = 0; u < ni; ++u)
              for (int v = 0; v < nj; ++v) {
                int I2 = Is[u], J2 = Js[v];
                if (I2 <= 0 || I2 >= C.n1) continue;  // Dirichlet coarse rows carry no correction
                int dI = I2 - I, dJ = J2 - J;
                if (dI < -1 || dI > 1 || dJ < -1 || dJ > 1) return false;
                C.at(st_slot(dI, dJ), I, J) += wr * ent[e].s * wi * wj;
              }
          }
        }
      }
    }
  return true;
}

}  // namespace

struct apic_sim {
  int precision = APIC_FP64;
  int n_inst = 0, n_pop = 0;
  std::vector<apic_config_t> cfg;
  std::vector<Inst> inst;
  std::vector<Pop> pop;
  cudaStream_t stream = nullptr;
  cudaStream_t cap = nullptr, cap2 = nullptr;
  apic_allocator_t alloc{};
  bool have_alloc = false;
  std::vector<void*> blocks;
  DevPtrs d{};
  SolvePlan plan{};
  cudaGraph_t graph[2] = {};
  cudaGraphExec_t exec[2] = {};       // one step graph per particle-buffer parity
  cudaGraph_t sort_graph[2] = {};
  cudaGraphExec_t sort_exec[2] = {};
  int par = 0;                        // which buffer holds the particles (1: the y arrays)
  int sort_interval = 0;
  long long host_step = 0;
  bool dirty = true;
  int status = APIC_OK;
  std::string msg = "ok";
  long long max_inj = 0;
  int push_grid = 0;
  int max_n2 = 0;                     // widest grid of the batch (cells in x2)
  int max_n1 = 0;                     // most cell rows of the batch (cells in x1)
  double* phi_save = nullptr;
  int32_t* h_err = nullptr;
  unsigned char* h_tally = nullptr;   // pinned staging of apic_tallies (the largest instance's copies)
  size_t h_tally_bytes = 0;
  bool cond_loop = true;              // Krylov loop as a graph while-node (else a fixed unrolled loop)
  int coop = 0;                       // CTAs of the cooperative whole-solve kernel (0: per-phase kernels)
  cudaGraphExec_t phase_exec[2][APIC_NPHASE] = {};
  cudaGraph_t phase_graph[2][APIC_NPHASE] = {};
  cudaEvent_t ev[APIC_NPHASE + 1] = {};
  double phase_ms[APIC_NPHASE] = {};
  long long timed_steps = 0;
  long long timed_sorts = 0;          // sorts inside apic_step_timed, and their CUDA-event time
  double sort_ms = 0.0;
  cudaEvent_t sort_ev[2] = {};
  long long slots = 0;                // particle slots of one buffer (all populations)
  long long sorts = 0;                // particle sorts launched
  size_t bcr_bytes = 0;               // reduction blocks + tail inverse (one device range)
  bool chord = false;                 // some instance absorbs grazing orbits (APIC_CHORD_ABSORB)
  bool floating = false;              // some instance has an isolated grain (APIC_FLOATING)
  bool boltz = false;                 // some instance has Boltzmann electrons (APIC_BOLTZMANN)
  int newton = 0;                     // Newton iterations per solve (the largest of those instances)
  double newton_eta = kNewtonEta;     // inexact-Newton reduction of every linear solve but the last
  size_t l2_persist = 0;              // bytes of L2 set aside for them (0: none)
  long long tab_total = 0;
  TanPtrs tan{};                      // sensitivity-window state (allocated on first use)
  bool tan_ready = false;
  int win_rows = 0;                   // push deposit window rows (0: default for the grid), set by apic_autotune
  int chunk_group = 0;                // push chunks per group (0: default), set by apic_autotune
  int chunk_items = 0;                // vector push particles per thread of a chunk (0: default), apic_autotune
  AdjPtrs adj{};                      // reverse-sweep state (allocated on first use, for up to adj_K steps)
  int adj_K = 0;
  std::vector<std::vector<std::pair<int, int>>> adj_levels;  // per instance, per tree level: fronts [f0, f1)
  std::vector<int> adj_smem;                                  // per instance: doubles of a front's vector

  int fail(int code, const std::string& m) {
    if (status == APIC_OK) {
      status = code;
      msg = m;
    }
    return status;
  }
  bool ck(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return true;
    fail(APIC_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
    return false;
  }
  void* dalloc(size_t bytes) {
    if (bytes == 0) bytes = 256;
    bytes = (bytes + 255) & ~(size_t)255;
    void* p = nullptr;
    if (have_alloc) {
      p = alloc.alloc(bytes, (void*)stream, alloc.ctx);
      if (!p) {
        fail(APIC_ERR_CUDA, "allocator returned NULL");
        return nullptr;
      }
    } else {
      if (!ck(cudaMallocAsync(&p, bytes, stream), "cudaMallocAsync")) return nullptr;
    }
    blocks.push_back(p);
    if (!ck(cudaMemsetAsync(p, 0, bytes, stream), "cudaMemsetAsync")) return nullptr;
    return p;
  }
  void dfree_all() {
    for (void* p : blocks) {
      if (have_alloc) alloc.free(p, (void*)stream, alloc.ctx);
      else cudaFreeAsync(p, stream);
    }
    blocks.clear();
  }
  template <class T>
  bool h2d(T* dst, const T* src, size_t n) {
    return ck(cudaMemcpyAsync(dst, src, n * sizeof(T), cudaMemcpyHostToDevice, stream), "H2D");
  }
  template <class T>
  bool d2h(T* dst, const T* src, size_t n) {
    return ck(cudaMemcpyAsync(dst, src, n * sizeof(T), cudaMemcpyDeviceToHost, stream), "D2H");
  }
  bool sync() { return ck(cudaStreamSynchronize(stream), "stream sync"); }
  // Device pointers with the particle buffers of parity p in front.
  DevPtrs view(int p) const {
    DevPtrs v = d;
    if (p) {
      std::swap(v.x1, v.y1);
      std::swap(v.x2, v.y2);
      std::swap(v.vR, v.yR);
      std::swap(v.vZ, v.yZ);
      std::swap(v.vT, v.yT);
    }
    return v;
  }
};

// After a set-up kernel with grid barriers: false (and APIC_ERR_TIMEOUT) if a
// barrier wait gave up.  Call after a synchronisation.
static bool setup_wait_ok(apic_sim* S, const char* what) {
  if (!S->d2h(S->h_err, S->d.err, 1) || !S->sync()) return false;
  if (*S->h_err & kErrTimeout) {
    S->fail(APIC_ERR_TIMEOUT, std::string(what) + ": grid barrier wait timed out");
    return false;
  }
  return true;
}

namespace {

int validate(const apic_config_t& c, std::string& why) {
  if (c.n1 < 4 || c.n2 < 8) return why = "n1 >= 4 and n2 >= 8 cells required", APIC_ERR_INVALID_ARG;
  if (c.n1 > 4096 || c.n2 > 2048) return why = "grid too large", APIC_ERR_INVALID_ARG;
  if (!(std::fabs(c.alpha) < 0.245)) return why = "|alpha| must be < 0.245 (closed grain, Eqs. 2-5)", APIC_ERR_GEOMETRY;
  if (!(c.x1_outer > -1.0 && c.x1_outer < 0.0)) return why = "x1_outer must lie in (-1, 0)", APIC_ERR_GEOMETRY;
  if (c.n_species < 1 || c.n_species > 2) return why = "n_species must be 1 or 2", APIC_ERR_INVALID_ARG;
  if (!(c.dt > 0.0)) return why = "dt must be > 0", APIC_ERR_INVALID_ARG;
  for (int s = 0; s < c.n_species; ++s) {
    const apic_species_t& p = c.sp[s];
    if (!(p.m > 0.0) || !(p.T >= 0.0) || p.n_init <= 0 || p.capacity <= 0 || p.capacity >= (1ll << 31))
      return why = "bad species parameters (m > 0, T >= 0, n_init > 0, 0 < capacity < 2^31)", APIC_ERR_INVALID_ARG;
  }
  if (c.precision != APIC_FP64 && c.precision != APIC_FP32_REFINED) return why = "bad precision", APIC_ERR_INVALID_ARG;
  if ((c.flags & (APIC_FLOATING | APIC_BOLTZMANN)) && (c.flags & APIC_NO_FIELD))
    return why = "APIC_FLOATING and APIC_BOLTZMANN need the field (not with APIC_NO_FIELD)", APIC_ERR_INVALID_ARG;
  if ((c.flags & APIC_FLOATING) && (c.flags & APIC_BOLTZMANN))
    return why = "APIC_FLOATING does not take APIC_BOLTZMANN (no electron current)", APIC_ERR_INVALID_ARG;
  if (c.newton_iters < 0 || c.newton_iters > 100) return why = "newton_iters in [0, 100]", APIC_ERR_INVALID_ARG;
  return APIC_OK;
}

// Inverse-CDF tables of x2 on [-1, 1]: volume dV/dx2 = (2 pi/3)(r_out^3 - r_g^3)
// (Eq. 5 integrated along x1) and dA/dx2 of Eq. 4 at x1_out; also the grain
// area.  Generic in the number type so that the sensitivity window can take
// the same sums on dual numbers.
template <class T>
void tables_t(const Inst& I, T alpha, std::vector<T>& tab, T& V_dom, T& A_out, T& A_grain) {
  const GL10& g = gl10();
  tab.assign(2 * (kTable + 1), T(0.0));
  T* cv = tab.data();
  T* cs = tab.data() + kTable + 1;
  double ht = 2.0 / kTable;
  T ag(0.0);
  for (int k = 0; k < kTable; ++k) {
    double lo = -1.0 + k * ht;
    T sv(0.0), ss(0.0), sg(0.0);
    for (int q = 0; q < 10; ++q) {
      double x2 = lo + 0.5 * (g.x[q] + 1.0) * ht, wq = 0.5 * g.w[q] * ht;
      T ro = radius(alpha, T(I.x1_out), T(x2)), rg = r_grain(alpha, T(x2));
      sv += T(wq) * T(2.0 * kPi / 3.0) * (ro * ro * ro - rg * rg * rg);
      ss += T(wq) * area_density(alpha, T(I.x1_out), T(x2));
      sg += T(wq) * area_density(alpha, T(-1.0), T(x2));
    }
    cv[k + 1] = cv[k] + sv;
    cs[k + 1] = cs[k] + ss;
    ag += sg;
  }
  V_dom = cv[kTable];
  A_out = cs[kTable];
  A_grain = ag;
}

void build_tables(Inst& I, std::vector<double>& tab) { tables_t<double>(I, I.alpha, tab, I.V_dom, I.A_out, I.A_grain); }

// Guide of each of the two tables: entry g holds the largest interval lo
// with cdf[lo] <= (g / kTable) * cdf[kTable] (the sampler scans forward from it).
std::vector<int32_t> guide_tables(const std::vector<double>& tab) {
  std::vector<int32_t> g(tab.size(), 0);
  for (int w = 0; w < 2; ++w) {
    const double* cdf = tab.data() + w * (kTable + 1);
    int32_t* out = g.data() + w * (kTable + 1);
    int lo = 0;
    for (int q = 0; q <= kTable; ++q) {
      double t = ((double)q / kTable) * cdf[kTable];
      while (lo + 1 < kTable && cdf[lo + 1] <= t) ++lo;
      out[q] = lo;
    }
  }
  return g;
}

// Geometry of the grain surface x1 = -1 at the x2 nodes (constant in time):
// |grad x1| and n_Z = (dx1/dZ) / |grad x1| from the metric of Eq. 2 at
// r_g(x2), dA/dx2 of Eq. 4, and the trapezoid weight.
std::vector<double> surface_geometry(const Inst& I) {
  std::vector<double> g(4 * (size_t)I.N2);
  for (int j = 0; j <= I.n2; ++j) {
    double x2 = x2_node_h(I, j);
    double r = r_grain(I.alpha, x2);
    Metric<double> m = metric(I.alpha, r, x2);
    double gn = std::sqrt(m.x1R * m.x1R + m.x1Z * m.x1Z);
    g[4 * j + 0] = gn;
    g[4 * j + 1] = m.x1Z / gn;
    g[4 * j + 2] = area_density(I.alpha, -1.0, x2);
    g[4 * j + 3] = (j == 0 || j == I.n2) ? 0.5 * I.h2 : I.h2;
  }
  return g;
}

// Hat-weighted node volumes: V_ij = integral over the (up to four) adjacent
// cells of the bilinear weight of node (i, j) times dOmega of Eq. 5.
template <class T>
void volumes_t(const Inst& I, T alpha, std::vector<T>& V) {
  const GL10& g = gl10();
  V.assign((size_t)I.nodes, T(0.0));
  for (int ci = 0; ci < I.n1; ++ci) {
    double xa = x1_node_h(I, ci), xb = x1_node_h(I, ci + 1);
    for (int cj = 0; cj < I.n2; ++cj) {
      double ya = x2_node_h(I, cj), yb = x2_node_h(I, cj + 1);
      T acc[4] = {T(0.0), T(0.0), T(0.0), T(0.0)};
      for (int a = 0; a < 10; ++a) {
        double f1 = 0.5 * (g.x[a] + 1.0), x1 = xa + f1 * (xb - xa);
        for (int b = 0; b < 10; ++b) {
          double f2 = 0.5 * (g.x[b] + 1.0), x2 = ya + f2 * (yb - ya);
          T wq = T(0.25 * g.w[a] * g.w[b] * (xb - xa) * (yb - ya)) * volume_density(alpha, T(x1), T(x2));
          acc[0] += wq * T(1.0 - f1) * T(1.0 - f2);
          acc[1] += wq * T(f1) * T(1.0 - f2);
          acc[2] += wq * T(1.0 - f1) * T(f2);
          acc[3] += wq * T(f1) * T(f2);
        }
      }
      V[(size_t)ci * I.N2 + cj] += acc[0];
      V[(size_t)(ci + 1) * I.N2 + cj] += acc[1];
      V[(size_t)ci * I.N2 + cj + 1] += acc[2];
      V[(size_t)(ci + 1) * I.N2 + cj + 1] += acc[3];
    }
  }
}

void build_volumes(const Inst& I, std::vector<double>& V) { volumes_t<double>(I, I.alpha, V); }

// Conservative form of Eqs. 6-7 (APIC_FE_OPERATOR): the weak form of Eq. 6
// with the bilinear hat functions N_a of the logical grid, which are also the
// charge-assignment weights, so that sum_b K_ab phi_b = rho_a V_a (Eq. 5's
// node volume) with
//   K_ab = int grad N_a . grad N_b dOmega = int J g^kl dN_a/dx_k dN_b/dx_l dx1 dx2,
// g^kl = grad x_k . grad x_l (the chain rule of Eq. 2) and J = dOmega/(dx1 dx2)
// (Eq. 5).  Cell (ci, cj), corner p = px + 2 py at node (ci + px, cj + py),
// integrated with 3 x 3 Gauss-Legendre points; in the two cells next to a
// pole the x2 points are placed in t with x2 = pole -+ h2 t^2, where J's
// sqrt(1 - x2^2) growth becomes smooth.
template <class T>
void fe_cell_h(const Inst& I, T alpha, int ci, int cj, T K[4][4]) {
  const double gx[3] = {-0.7745966692414834, 0.0, 0.7745966692414834};  // +-sqrt(3/5), 0
  const double gw[3] = {5.0 / 9.0, 8.0 / 9.0, 5.0 / 9.0};
  const double xa = x1_node_h(I, ci), xb = x1_node_h(I, ci + 1);
  const double ya = x2_node_h(I, cj), yb = x2_node_h(I, cj + 1);
  for (int p = 0; p < 4; ++p)
    for (int q = 0; q < 4; ++q) K[p][q] = T(0.0);
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      const double f1 = 0.5 * (gx[a] + 1.0), x1 = xa + f1 * (xb - xa);
      double wq = 0.25 * gw[a] * gw[b] * (xb - xa) * (yb - ya);
      double f2 = 0.5 * (gx[b] + 1.0), x2;
      if (cj == 0) {  // x2 = -1 + h2 t^2, dx2 = 2 h2 t dt
        x2 = ya + (yb - ya) * f2 * f2;
        wq *= 2.0 * f2;
        f2 = f2 * f2;
      } else if (cj == I.n2 - 1) {  // x2 = 1 - h2 t^2
        const double t = f2;
        x2 = yb - (yb - ya) * t * t;
        wq *= 2.0 * t;
        f2 = 1.0 - t * t;
      } else {
        x2 = ya + f2 * (yb - ya);
      }
      const Metric<T> m = metric(alpha, radius(alpha, T(x1), T(x2)), T(x2));
      const T g11 = m.x1R * m.x1R + m.x1Z * m.x1Z, g22 = m.x2R * m.x2R + m.x2Z * m.x2Z;
      const T g12 = m.x1R * m.x2R + m.x1Z * m.x2Z;
      const T Jw = volume_density(alpha, T(x1), T(x2)) * T(wq);
      double d1[4], d2[4];  // derivatives of the corner functions at (f1, f2)
      for (int p = 0; p < 4; ++p) {
        const int px = p & 1, py = p >> 1;
        const double sx = px ? 1.0 : -1.0, sy = py ? 1.0 : -1.0;
        const double ex = px ? f1 : 1.0 - f1, ey = py ? f2 : 1.0 - f2;
        d1[p] = sx * ey / (xb - xa);
        d2[p] = sy * ex / (yb - ya);
      }
      for (int p = 0; p < 4; ++p)
        for (int q = 0; q < 4; ++q)
          K[p][q] += Jw * (g11 * T(d1[p] * d1[q]) + g12 * T(d1[p] * d2[q] + d2[p] * d1[q]) + g22 * T(d2[p] * d2[q]));
    }
}

// Row (i, j) of the discrete operator, unscaled, in the form L phi = -rho:
// the kSt stencil weights (Dirichlet neighbours included).  Eq. 7 with
// second-order differences, or with APIC_FE_OPERATOR the conservative form's
// row -K_a / V_a (V: the node volumes).  Returns a1 = A / h1^2 of Eq. 7, the
// row scale of both forms.
template <class T>
T fine_row(const Inst& I, T alpha, int i, int j, T w[kSt], const T* V) {
  LapCoef<T> c = lap_coef(alpha, T(x1_node_h(I, i)), T(x2_node_h(I, j)));
  T a1 = c.A / T(I.h1 * I.h1);
  for (int k = 0; k < kSt; ++k) w[k] = T(0.0);
  if (I.flags & APIC_FE_OPERATOR) {
    const T Va = V[(size_t)i * I.N2 + j];
    for (int ci = i - 1; ci <= i; ++ci)
      for (int cj = j - 1; cj <= j; ++cj) {
        if (ci < 0 || ci >= I.n1 || cj < 0 || cj >= I.n2) continue;
        T K[4][4];
        fe_cell_h<T>(I, alpha, ci, cj, K);
        const int pa = (i - ci) | ((j - cj) << 1);
        for (int q = 0; q < 4; ++q) w[st_slot(ci + (q & 1) - i, cj + (q >> 1) - j)] -= K[pa][q] / Va;
      }
    return a1;
  }
  w[st_slot(-1, 0)] += a1;
  w[st_slot(1, 0)] += a1;
  w[st_slot(0, 0)] += T(-2.0) * a1;
  T e = c.E / T(2.0 * I.h2);
  if (j == 0) {
    w[st_slot(0, 0)] += T(-3.0) * e;
    w[st_slot(0, 1)] += T(4.0) * e;
    w[kStPole] += T(-1.0) * e;
  } else if (j == I.n2) {
    w[st_slot(0, 0)] += T(3.0) * e;
    w[st_slot(0, -1)] += T(-4.0) * e;
    w[kStPole] += T(1.0) * e;
  } else {
    T a2 = c.C / T(I.h2 * I.h2), dd = c.D / T(4.0 * I.h1 * I.h2);
    w[st_slot(0, -1)] += a2 - e;
    w[st_slot(0, 1)] += a2 + e;
    w[st_slot(0, 0)] += T(-2.0) * a2;
    w[st_slot(1, 1)] += dd;
    w[st_slot(-1, -1)] += dd;
    w[st_slot(1, -1)] -= dd;
    w[st_slot(-1, 1)] -= dd;
  }
  return a1;
}

// Finest-level operator (fine_row), each row scaled by rscale = 1/a1 =
// h1^2 / A; entries towards the Dirichlet rows are moved to bbc (times phi_g
// or phi_out) and stored as zero.
void build_fine(const Inst& I, const std::vector<double>& V, HostLevel& L, std::vector<double>& rscale,
                std::vector<double>& bbc) {
  L.n1 = I.n1;
  L.n2 = I.n2;
  L.N1 = I.N1;
  L.N2 = I.N2;
  L.st.assign((size_t)kSt * L.nodes(), 0.0);
  rscale.assign((size_t)I.nodes, 0.0);
  bbc.assign((size_t)I.nodes, 0.0);
  for (int i = 1; i < I.n1; ++i)
    for (int j = 0; j <= I.n2; ++j) {
      double w[kSt];
      double a1 = fine_row<double>(I, I.alpha, i, j, w, V.data());
      double sc = 1.0 / a1;
      size_t nd = (size_t)i * I.N2 + j;
      rscale[nd] = sc;
      double bb = 0.0;
      for (int k = 0; k < kSt; ++k) w[k] *= sc;
      for (int dj = -1; dj <= 1; ++dj) {
        if (i == 1) {
          bb -= w[st_slot(-1, dj)] * I.phi_g;
          w[st_slot(-1, dj)] = 0.0;
        }
        if (i == I.n1 - 1) {
          bb -= w[st_slot(1, dj)] * I.phi_out;
          w[st_slot(1, dj)] = 0.0;
        }
      }
      bbc[nd] = bb;
      for (int k = 0; k < kSt; ++k) L.at(k, i, j) = w[k];
    }
}

// The Dirichlet term of the problem with phi = 1 on the grain and 0 on the
// outer surface, rows scaled as build_fine's (nonzero on the row i = 1 only).
void grain_bbc(const Inst& I, std::vector<double>& hbg) {
  std::vector<double> V;
  build_volumes(I, V);
  hbg.assign((size_t)I.nodes, 0.0);
  for (int j = 0; j <= I.n2; ++j) {
    double w[kSt];
    double sc = 1.0 / fine_row<double>(I, I.alpha, 1, j, w, V.data());
    double bb = 0.0;
    for (int dj = -1; dj <= 1; ++dj) bb -= w[st_slot(-1, dj)] * sc;
    hbg[(size_t)I.N2 + j] = bb;
  }
}

// ---- block cyclic reduction set-up (FP64 on the host, blocks stored in FP32) ----
using Mat = std::vector<double>;  // row-major n x n

// c = a b; zeros of a are skipped and each row of b is visited over its
// nonzero range only, so products with the tridiagonal blocks of Eq. 7 cost
// O(n^2).
void mat_mul(const Mat& a, const Mat& b, Mat& c, int n) {
  c.assign((size_t)n * n, 0.0);
  std::vector<int> lo(n), hi(n);
  for (int k = 0; k < n; ++k) {
    const double* bk = b.data() + (size_t)k * n;
    int l = 0, h = n - 1;
    while (l < n && bk[l] == 0.0) ++l;
    while (h >= l && bk[h] == 0.0) --h;
    lo[k] = l;
    hi[k] = h;
  }
  for (int i = 0; i < n; ++i) {
    double* ci = c.data() + (size_t)i * n;
    for (int k = 0; k < n; ++k) {
      double aik = a[(size_t)i * n + k];
      if (aik == 0.0 || lo[k] > hi[k]) continue;
      const double* bk = b.data() + (size_t)k * n;
      for (int j = lo[k]; j <= hi[k]; ++j) ci[j] += aik * bk[j];
    }
  }
}

// Gauss-Jordan elimination with partial pivoting; false if singular.
bool mat_inv(const Mat& a, Mat& inv, int n) {
  Mat w(a);
  inv.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) inv[(size_t)i * n + i] = 1.0;
  for (int c = 0; c < n; ++c) {
    int p = c;
    double best = std::fabs(w[(size_t)c * n + c]);
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(w[(size_t)r * n + c]) > best) {
        best = std::fabs(w[(size_t)r * n + c]);
        p = r;
      }
    if (!(best > 0.0)) return false;
    if (p != c)
      for (int j = 0; j < n; ++j) {
        std::swap(w[(size_t)c * n + j], w[(size_t)p * n + j]);
        std::swap(inv[(size_t)c * n + j], inv[(size_t)p * n + j]);
      }
    double s = 1.0 / w[(size_t)c * n + c];
    for (int j = 0; j < n; ++j) {
      w[(size_t)c * n + j] *= s;
      inv[(size_t)c * n + j] *= s;
    }
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      double f = w[(size_t)r * n + c];
      if (f == 0.0) continue;
      for (int j = 0; j < n; ++j) {
        w[(size_t)r * n + j] -= f * w[(size_t)c * n + j];
        inv[(size_t)r * n + j] -= f * inv[(size_t)c * n + j];
      }
    }
  }
  return true;
}

template <class F>
void parallel_for(int n, F f) {
  int T = (int)std::min<unsigned>(16u, std::max(1u, std::thread::hardware_concurrency()));
  T = std::min(T, n);
  if (T <= 1) {
    for (int q = 0; q < n; ++q) f(q);
    return;
  }
  std::vector<std::thread> th;
  for (int t = 0; t < T; ++t)
    th.emplace_back([&, t] {
      for (int q = t; q < n; q += T) f(q);
    });
  for (auto& x : th) x.join();
}

double nd_coef(const void* ctx, int i, int j, int slot) { return ((const HostLevel*)ctx)->get(slot, i, j); }

// Layout of instance I's reduction: block size, levels before the dense
// tail, first block of each kind per level (real rows only).  False if the
// reduction does not apply (N2 > kBcrMaxNWide, n1 < 4, n1 > 2^(kBcrMaxK-1)).
bool bcr_layout(const Inst& I, BcrInst& bp, bool dense1) {
  std::memset(&bp, 0, sizeof(bp));
  bp.dense1 = dense1 ? 1 : 0;
  const int N = I.N2, M = I.n1 - 1;
  if (I.n1 < 4 || N > kBcrMaxNWide) return false;
  int K = 0;
  while ((1 << K) < I.n1) ++K;
  if (K >= kBcrMaxK) return false;
  int Lt = 0;
  while (Lt < K - 1 && (long long)(M >> Lt) * N > kBcrTailMax) ++Lt;
  if (const char* e = std::getenv("APIC_BCR_LEVELS")) {  // tuning: more reduction levels, smaller tail
    int v = std::atoi(e);
    if (v >= Lt && v <= K - 1) Lt = v;
  }
  long long nblk = 0;
  for (int l = 1; l <= Lt; ++l) {
    const int h = 1 << (l - 1);
    const long long ne = (M / h + 1) / 2, nk = M / (2 * h);
    if (l == 1 && !dense1) {
      bp.Binv[l] = nblk;
      nblk += ne;
      continue;
    }
    bp.P[l] = nblk;
    nblk += nk;
    bp.Q[l] = nblk;
    nblk += nk;
    bp.Binv[l] = nblk;
    nblk += ne;
    bp.G[l] = nblk;
    nblk += ne;
    bp.H[l] = nblk;
    nblk += ne;
  }
  bp.blocks = nblk;
  bp.K = K;
  bp.N = N;
  bp.Np = (N + 3) & ~3;
  bp.blk = (long long)N * bp.Np;
  bp.Lt = Lt;
  bp.M = M;
  bp.tail_m = M >> Lt;
  bp.tail_n = bp.tail_m * N;
  bp.tail_np = (bp.tail_n + 3) & ~3;
  return bp.tail_n <= kBcrTailMax;
}

// Blocks of the reduction of instance I's finest-level system (stencil of
// level L, rows scaled, Dirichlet neighbours zero) in the layout bp, and the
// dense tail system T (FP64, row-major, inverted on the GPU by the caller);
// false if a pivot vanishes.
bool bcr_factor(const HostLevel& L, const BcrInst& bp, std::vector<float>& out, std::vector<double>& T) {
  const int N = bp.N, M = bp.M, Np = bp.Np, Lt = bp.Lt;
  std::vector<Mat> A(M + 2), Bm(M + 2), C(M + 2);
  parallel_for(M, [&](int r) {
    const int i = r + 1;
    A[i].assign((size_t)N * N, 0.0);
    Bm[i].assign((size_t)N * N, 0.0);
    C[i].assign((size_t)N * N, 0.0);
    for (int j = 0; j < N; ++j) {
      for (int dj = -1; dj <= 1; ++dj) {
        int jj = j + dj;
        if (jj < 0 || jj >= N) continue;
        A[i][(size_t)j * N + jj] = L.get(st_slot(-1, dj), i, j);
        Bm[i][(size_t)j * N + jj] = L.get(st_slot(0, dj), i, j);
        C[i][(size_t)j * N + jj] = L.get(st_slot(1, dj), i, j);
      }
    }
    Bm[i][2] += L.get(kStPole, i, 0);
    Bm[i][(size_t)(N - 1) * N + N - 3] += L.get(kStPole, i, N - 1);
  });
  out.assign((size_t)std::max<long long>(1, bp.blocks) * bp.blk, 0.0f);
  auto store = [&](long long idx, const Mat& m) {
    float* o = out.data() + (size_t)idx * bp.blk;
    for (int r = 0; r < N; ++r)
      for (int c = 0; c < N; ++c) o[(size_t)c * Np + r] = (float)m[(size_t)r * N + c];
  };
  bool ok = true;
  for (int l = 1; l <= Lt && ok; ++l) {
    const int h = 1 << (l - 1), ne = (M / h + 1) / 2, nk = M / (2 * h);
    std::vector<Mat> Binv(ne);
    std::vector<char> good(ne, 1);
    parallel_for(ne, [&](int q) {
      const int k = h * (2 * q + 1);
      if (!mat_inv(Bm[k], Binv[q], N)) {
        good[q] = 0;
        return;
      }
      store(bp.Binv[l] + q, Binv[q]);
      if (l == 1 && !bp.dense1) return;  // level 1 applies A_k and C_k from the stencil
      Mat t;
      mat_mul(Binv[q], A[k], t, N);
      store(bp.G[l] + q, t);
      mat_mul(Binv[q], C[k], t, N);
      store(bp.H[l] + q, t);
    });
    for (char g : good) ok = ok && g;
    if (!ok) break;
    std::vector<Mat> nA(nk), nB(nk), nC(nk);
    parallel_for(nk, [&](int q) {
      const int i = 2 * h * (q + 1);
      const bool right = i + h <= M;  // else C_i = 0: row i + h carries no unknowns
      Mat P, Q, t;
      mat_mul(A[i], Binv[q], P, N);
      if (right) mat_mul(C[i], Binv[q + 1], Q, N);
      else Q.assign((size_t)N * N, 0.0);
      if (l > 1 || bp.dense1) {
        store(bp.P[l] + q, P);
        store(bp.Q[l] + q, Q);
      }
      mat_mul(P, A[i - h], t, N);
      nA[q].assign((size_t)N * N, 0.0);
      for (size_t e = 0; e < t.size(); ++e) nA[q][e] = -t[e];
      nC[q].assign((size_t)N * N, 0.0);
      nB[q] = Bm[i];
      mat_mul(P, C[i - h], t, N);
      for (size_t e = 0; e < t.size(); ++e) nB[q][e] -= t[e];
      if (right) {
        mat_mul(Q, C[i + h], t, N);
        for (size_t e = 0; e < t.size(); ++e) nC[q][e] = -t[e];
        mat_mul(Q, A[i + h], t, N);
        for (size_t e = 0; e < t.size(); ++e) nB[q][e] -= t[e];
      }
    });
    // the eliminated rows are no longer needed
    for (int q = 0; q < ne; ++q) {
      const int k = h * (2 * q + 1);
      Mat().swap(A[k]);
      Mat().swap(Bm[k]);
      Mat().swap(C[k]);
    }
    for (int q = 0; q < nk; ++q) {
      const int i = 2 * h * (q + 1);
      A[i].swap(nA[q]);
      Bm[i].swap(nB[q]);
      C[i].swap(nC[q]);
    }
  }
  if (!ok) return false;
  // the rows left, i = 2^Lt (q + 1) <= M: dense block tridiagonal system
  const int m = bp.tail_m, n = bp.tail_n, hs = 1 << Lt;
  T.assign((size_t)n * n, 0.0);
  for (int q = 0; q < m; ++q) {
    const int i = hs * (q + 1);
    for (int r = 0; r < N; ++r)
      for (int c = 0; c < N; ++c) {
        size_t row = (size_t)q * N + r;
        T[row * n + (size_t)q * N + c] = Bm[i][(size_t)r * N + c];
        if (q > 0) T[row * n + (size_t)(q - 1) * N + c] = A[i][(size_t)r * N + c];
        if (q < m - 1) T[row * n + (size_t)(q + 1) * N + c] = C[i][(size_t)r * N + c];
      }
  }
  return true;
}

}  // namespace

// ---------------------------------------------------------------------------
// Creation.
// ---------------------------------------------------------------------------
template <class Real>
static bool vacuum_fields(apic_sim* S);

template <class Real>
static int setup(apic_sim* S) {
  const int ni = S->n_inst;
  std::vector<std::vector<double>> tabs(ni), vols(ni), rscs(ni), bbcs(ni);
  std::vector<std::vector<HostLevel>> levels(ni);
  std::vector<std::vector<double>> cinvs(ni);
  long long total_nodes = 0, level_nodes = 0, tab_total = 0, bins_total = 0, hist_total = 0, en_total = 0,
            cinv_total = 0, slots = 0, total_cells = 0, fac_total = 0;
  int pop_index = 0;
  for (int k = 0; k < ni; ++k) {
    const apic_config_t& c = S->cfg[k];
    Inst I;
    std::memset(&I, 0, sizeof(I));
    I.alpha = c.alpha;
    I.x1_out = c.x1_outer;
    I.phi_g = c.phi_grain;
    I.phi_out = c.phi_outer;
    I.B = c.B;
    I.dt = c.dt;
    I.e_bind = c.e_bind_ion;
    I.n1 = c.n1;
    I.n2 = c.n2;
    I.N1 = c.n1 + 1;
    I.N2 = c.n2 + 1;
    I.h1 = (c.x1_outer + 1.0) / c.n1;
    I.h2 = 2.0 / c.n2;
    I.i2h1 = 1.0 / (2.0 * I.h1);
    I.i2h2 = 1.0 / (2.0 * I.h2);
    I.nodes = (long long)I.N1 * I.N2;
    I.node_off = total_nodes;
    total_nodes += I.nodes;
    I.tol = c.poisson_tol > 0 ? c.poisson_tol : 1e-10;
    I.max_iter = c.poisson_max_iter > 0 ? c.poisson_max_iter : 20;
    I.seed = c.seed;
    I.tag = c.instance;
    I.flags = c.flags;
    I.guess = c.poisson_guess == 1 ? 1 : 0;
    I.n_species = c.n_species;
    I.pop0 = pop_index;
    I.hist_cap = c.history_cap > 0 ? c.history_cap : 4096;
    I.tab_off = tab_total;
    tab_total += 2 * (kTable + 1);
    I.bin_off = bins_total;
    bins_total += (long long)c.n_species * ((long long)c.n2 * kTallyBinWords + kTallyStepWords);
    I.hist_off = hist_total;
    hist_total += (long long)I.hist_cap * kNH;
    I.en_off = en_total;
    en_total += I.N2;
    build_tables(I, tabs[k]);
    build_volumes(I, vols[k]);
    // operator and multigrid hierarchy
    levels[k].emplace_back();
    build_fine(I, vols[k], levels[k][0], rscs[k], bbcs[k]);
    while (true) {
      const HostLevel& F = levels[k].back();
      if ((int)levels[k].size() >= kMaxLevels) break;
      if ((long long)(F.n1 - 1) * F.N2 <= kMaxCoarse) break;
      if (F.n1 % 2 || F.n2 % 2 || F.n1 < 8 || F.n2 < 4) break;
      HostLevel C;
      if (!galerkin(F, C, levels[k].size() == 1)) return S->fail(APIC_ERR_INVALID_ARG, "coarse stencil wider than 3x3");
      levels[k].push_back(std::move(C));
    }
    I.n_levels = (int)levels[k].size();
    // every level but the coarsest is smoothed; the coarsest is solved with its dense inverse
    I.tail_level = I.n_levels - 1;
    for (int l = 0; l < I.n_levels; ++l) {
      Level& L = I.lv[l];
      const HostLevel& H = levels[k][l];
      L.n1 = H.n1;
      L.n2 = H.n2;
      L.N1 = H.N1;
      L.N2 = H.N2;
      L.off = level_nodes;
      L.st = (long long)kSt * level_nodes;
      L.pole_extra = l == 0 ? 1 : 0;
      level_nodes += H.nodes();
      int k1 = (H.n1 - 1 + 31) / 32, k2 = (H.n2 + 1 + 31) / 32;
      L.fac[0] = fac_total;
      fac_total += (long long)H.N2 * line_fac_stride(k1);
      L.fac[1] = fac_total;
      fac_total += (long long)H.N1 * line_fac_stride(k2);
    }
    // coarsest dense inverse over rows 1..n1-1
    {
      const HostLevel& H = levels[k].back();
      int nu = (H.n1 - 1) * H.N2;
      if (nu > kMaxDense) return S->fail(APIC_ERR_INVALID_ARG, "coarsest multigrid level too large (grid not divisible)");
      std::vector<double> A((size_t)nu * nu, 0.0);
      for (int i = 1; i < H.n1; ++i)
        for (int j = 0; j <= H.n2; ++j) {
          int r = (i - 1) * H.N2 + j;
          for (int di = -1; di <= 1; ++di)
            for (int dj = -1; dj <= 1; ++dj) {
              int i2 = i + di, j2 = j + dj;
              if (i2 < 1 || i2 > H.n1 - 1 || j2 < 0 || j2 > H.n2) continue;
              A[(size_t)r * nu + (i2 - 1) * H.N2 + j2] += H.get(st_slot(di, dj), i, j);
            }
          if (I.n_levels == 1) {
            double s = H.get(kStPole, i, j);
            if (j == 0) A[(size_t)r * nu + (i - 1) * H.N2 + 2] += s;
            if (j == H.n2) A[(size_t)r * nu + (i - 1) * H.N2 + H.n2 - 2] += s;
          }
        }
      cinvs[k] = std::move(A);  // inverted on the GPU below
      I.coarse_n = nu;
      I.cinv_off = cinv_total;
      cinv_total += (long long)nu * nu;
    }
    for (int s = 0; s < c.n_species; ++s) {
      Pop P;
      std::memset(&P, 0, sizeof(P));
      const apic_species_t& sp = c.sp[s];
      P.q = sp.q;
      P.m = sp.m;
      P.T = sp.T;
      P.w = I.V_dom / (double)sp.n_init;
      P.vth = std::sqrt(sp.T / sp.m);
      P.tunit = P.vth;
      P.tfix_off = I.bin_off + (long long)s * ((long long)c.n2 * kTallyBinWords + kTallyStepWords);
      P.lam = std::sqrt(sp.T / (2.0 * kPi * sp.m)) * I.A_out * c.dt / P.w;
      P.base = slots;
      P.cap = sp.capacity;
      slots += (sp.capacity + 3) & ~3ll;  // slot ranges on 16-byte boundaries (the FP32 push's vector loads)
      P.inst = k;
      P.species = s;
      int lg = bits_for(sp.capacity);
      if (sizeof(Real) == 8) P.fbits = 62 - lg;
      else P.fbits = 2 * std::min(16, (62 - lg) / 2);  // 16-bit cell fractions (the push's packed moments)
      P.dep_scale = sp.q * P.w * std::ldexp(1.0, -P.fbits);
      P.acc_off = 2 * I.node_off + (long long)s * I.nodes;
      P.cells = c.n1;  // sort bins: the grid rows of this population
      P.cell_off = total_cells;
      total_cells += P.cells;
      S->max_inj = std::max(S->max_inj, (long long)std::ceil(P.lam) + 2);
      S->pop.push_back(P);
      ++pop_index;
    }
    S->inst.push_back(I);
  }
  S->n_pop = pop_index;
  S->slots = slots;
  S->tab_total = tab_total;
  if (S->n_pop > kMaxPop) return S->fail(APIC_ERR_INVALID_ARG, "too many instances x species");

  // ---- launch plan ----
  SolvePlan& pl = S->plan;
  std::memset(&pl, 0, sizeof(pl));
  for (const Inst& I : S->inst) pl.max_tail = std::max(pl.max_tail, I.tail_level);
  for (int l = 0; l < kMaxLevels; ++l) {
    int x1l = 0, x2l = 0, k1 = 1, k2 = 1;
    long long nodes = 1;
    for (const Inst& I : S->inst) {
      if (l >= I.n_levels) continue;
      const Level& L = I.lv[l];
      x1l = std::max(x1l, (L.n2 + 2) / 2);
      x2l = std::max(x2l, L.n1 / 2);
      k1 = std::max(k1, (L.n1 - 1 + 31) / 32);
      k2 = std::max(k2, (L.n2 + 1 + 31) / 32);
      nodes = std::max(nodes, (long long)L.N1 * L.N2);
    }
    pl.x1_blocks[l] = std::max(1, x1l);
    pl.x2_blocks[l] = std::max(1, x2l);
    pl.x1_k[l] = k1;
    pl.x2_k[l] = k2;
    pl.node_blocks[l] = (int)std::min<long long>(1024, std::max<long long>(1, (nodes + 255) / 256));
  }
  pl.tail_threads = 512;
  pl.tail_k = 1;
  pl.tail_bytes = 0;
  // x1-lines before restriction, x2-lines after prolongation: more Krylov
  // iterations than smoothing both ways twice, but fewer phases per step
  pl.smooth_split = 1;
  if (const char* sm = std::getenv("APIC_MG_SMOOTH")) pl.smooth_split = std::string(sm) != "alt";
  if (!S->ck(set_poisson_smem<Real>(pl), "cudaFuncSetAttribute(smem)")) return S->status;
  // Direct block cyclic reduction in place of multigrid: FP32 particles, every
  // instance with a field, N2 <= kBcrMaxNWide, the blocks of the batch within the
  // memory budget (APIC_PRECOND=mg keeps multigrid).
  std::vector<BcrInst> bcr_in;
  std::vector<int32_t> bcr_kind, bcr_pre, bcr_npre, bcr_tpre;
  long long bcr_rows = 0;  // floats of bcr_f (and of bcr_e)
  int bcr_nb = 0;          // CTAs of the reduction solve
  // nested dissection per instance (APIC_DIRECT=nd: every instance, bcr:
  // none, wide: grids wider than kBcrMaxN cells in x2; default: every
  // instance unless the whole reduction fits in L2)
  std::vector<NdFactor> nds(ni);
  std::vector<char> use_nd(ni, 0);
  NdUpload ndu;
  std::vector<int2> nd_flow;      // the dataflow sweeps' task orders
  std::vector<int32_t> nd_need;   // tasks per front and sweep
  long long nd_w = 0;  // floats of one right-hand side's update vectors
  {
    const char* pc = std::getenv("APIC_PRECOND");
    bool want = sizeof(Real) == 4 && ni <= kCoopMaxInst && !(pc && std::string(pc) == "mg");
    for (const Inst& I : S->inst) want = want && !(I.flags & (APIC_NO_FIELD | APIC_BOLTZMANN));
    const char* dm = std::getenv("APIC_DIRECT");
    const std::string direct = dm ? dm : "auto";
    // auto: the reduction where all its blocks (dense level 1) fit in L2
    // (fewer, shorter phases), else nested dissection (its fronts stream
    // about a tenth of the reduction's bytes from DRAM)
    bool red_fits = false;
    if (want && direct == "auto") {
      double b = 0.0;
      bool ok = true;
      for (int k = 0; k < ni && ok; ++k) {
        BcrInst B{};
        ok = bcr_layout(S->inst[k], B, true);
        b += 4.0 * ((double)B.blocks * (double)B.blk + (double)B.tail_n * (double)B.tail_np);
      }
      red_fits = ok && b <= 112.0 * 1024 * 1024;
    }
    for (int k = 0; k < ni && want; ++k) {
      const Inst& I = S->inst[k];
      // wide: nested dissection only where the narrow reduction does not
      // apply (a batch may then mix both in one launch)
      use_nd[k] = direct == "nd" || (direct == "auto" && !red_fits) || (direct == "wide" && I.N2 > kBcrMaxN + 1);
      if (!use_nd[k]) continue;
      std::string why;
      int T = (int)std::min<unsigned>(16u, std::max(1u, std::thread::hardware_concurrency()));
      static int leaf = -1;  // nodes per leaf piece at most (APIC_ND_LEAF, default 16)
      if (leaf < 0) {
        const char* e = std::getenv("APIC_ND_LEAF");
        leaf = e ? std::max(1, std::min(256, std::atoi(e))) : 16;
      }
      if (!nd_build(I.n1 - 1, I.N2, nd_coef, &levels[k][0], leaf, T, false, nds[k], why) ||
          nds[k].depth > kNdMaxDepth)
        use_nd[k] = 0;  // the reduction (or multigrid) instead
    }
    long long off = 0;
    // dense level-1 blocks when the whole reduction then still fits in L2
    // (fewer phases); else level 1 applies the stencil's couplings (fewer
    // bytes streamed from DRAM)
    const double l2_fit = 112.0 * 1024 * 1024;
    for (int dense1 = 1; dense1 >= 0 && want; --dense1) {
      off = 0;
      bcr_rows = 0;
      bcr_in.assign(ni, BcrInst{});
      ndu = NdUpload();
      nd_w = 0;
      int nd_need = 0;
      int sms = 0;  // CTAs of the solve: an instance's small fronts are spread over its share
      {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      }
      double nd_nodes = 0.0;
      for (int k = 0; k < ni; ++k)
        if (use_nd[k]) nd_nodes += (double)S->inst[k].nodes;
      for (int k = 0; k < ni && want; ++k) {
        BcrInst& B = bcr_in[k];
        auto up = [](long long v) { return (v + 63) & ~63ll; };  // 256-byte aligned ranges
        if (use_nd[k]) {
          std::memset(&B, 0, sizeof(B));
          const Inst& I = S->inst[k];
          B.M = I.n1 - 1;
          B.N = I.N2;
          B.Np = (B.N + 3) & ~3;
          B.base = off;
          NdLevels lvl;
          // the share of the CTAs by nodes (the sums do not depend on the
          // task layout: an instance computes the same alone or in a batch)
          const int nd_ctas = std::max(1, (int)std::lround(sms * (double)I.nodes / nd_nodes));
          nd_need = std::max(nd_need, nd_layout(nds[k], off, nd_w, kNdWarpMaxS, kNdWarpMaxU, kNdWarpStage, kNdTaskFloats,
                                                kNdTaskRows, kNdTaskFronts, kNdUnitStage, kNdUnits * nd_ctas,
                                                ndu, lvl));
          B.nd = 1;
          B.nd_depth = nds[k].depth;
          for (int l = 0; l <= nds[k].depth + 1; ++l) {
            B.nd_ft[l] = lvl.ft[l];
            B.nd_bt[l] = lvl.bt[l];
          }
          off += up(nds[k].fm_total + nds[k].nb_total);
          nd_w += up(nds[k].w_total);
          B.foff = bcr_rows;
          bcr_rows += (long long)B.M * B.N;
          B.node_off = I.node_off;
          B.nodes = I.nodes;
          B.st_off = I.lv[0].st;
          continue;
        }
        if (!bcr_layout(S->inst[k], B, dense1 != 0)) {
          want = false;
          break;
        }
        B.base = off;
        off += up(B.blocks * B.blk);
        B.tail = off;
        off += up((long long)B.tail_n * B.tail_np);
        B.foff = bcr_rows;
        bcr_rows += (long long)B.M * B.N;
        B.node_off = S->inst[k].node_off;
        B.nodes = S->inst[k].nodes;
        B.st_off = S->inst[k].lv[0].st;
      }
      pl.bcr.nd_floats = nd_need;
      if (4.0 * (double)off <= l2_fit) break;
    }
    const double bytes = 4.0 * (double)off;
    if (want) {
      size_t fr = 0, tot = 0;
      if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) fr = 0;
      cudaGetLastError();
      want = bytes <= kBcrMaxBytes && bytes <= 0.6 * (double)fr;
    }
    if (want) {
      int dev = 0, sms = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      pl.bcr.bytes = (int64_t)(4 * off);
      pl.bcr.resident = bytes <= l2_fit ? 1 : 0;  // the whole reduction fits in L2 (blocks are staged)
      want = (bcr_nb = bcr_configure(pl, bcr_in.data(), ni, sms)) > 0;  // else not co-residable: multigrid
    }
    if (want) {
      // stages of each instance, aligned at the first phase
      std::vector<std::vector<std::pair<int, int>>> stages(ni);  // (kind << 8 | level, tasks)
      int phases = 0;
      for (int k = 0; k < ni; ++k) {
        const BcrInst& B = bcr_in[k];
        auto& st = stages[k];
        const int M = B.M;
        auto ne = [&](int l) { return (M / (1 << (l - 1)) + 1) / 2; };
        auto nk = [&](int l) { return M / (2 << (l - 1)); };
        if (B.nd) {  // forward from the deepest level, then backward from the root
          for (int l = B.nd_depth; l >= 0; --l) st.push_back({kNdFwd << 8 | l, B.nd_ft[l + 1] - B.nd_ft[l]});
          for (int l = 0; l <= B.nd_depth; ++l) st.push_back({kNdBack << 8 | l, B.nd_bt[l + 1] - B.nd_bt[l]});
          phases = std::max(phases, (int)st.size());
          continue;
        }
        const int l0 = B.dense1 ? 1 : 2;  // first level with dense blocks
        if (B.Lt >= 1 && !B.dense1) {
          st.push_back({kBcrFwd1 << 8 | 1, ne(1)});
          st.push_back({kBcrUpd1 << 8 | 1, (nk(1) + kBcrUpdRows - 1) / kBcrUpdRows});
        }
        for (int l = l0; l <= B.Lt; ++l) st.push_back({kBcrFwd << 8 | l, nk(l)});
        st.push_back({kBcrTail << 8, (B.tail_n + B.tail_rows - 1) / B.tail_rows});
        for (int l = B.Lt; l >= l0; --l) st.push_back({kBcrBack << 8 | l, ne(l)});
        if (B.Lt >= 1 && !B.dense1) st.push_back({kBcrBack1 << 8 | 1, ne(1)});
        phases = std::max(phases, (int)st.size());
      }
      bcr_kind.assign((size_t)phases * ni, 0);
      bcr_pre.assign((size_t)phases * (ni + 1), 0);
      for (int p = 0; p < phases; ++p)
        for (int k = 0; k < ni; ++k) {
          int cnt = 0;
          if (p < (int)stages[k].size()) {
            bcr_kind[(size_t)p * ni + k] = stages[k][p].first;
            cnt = stages[k][p].second;
          }
          bcr_pre[(size_t)p * (ni + 1) + k + 1] = bcr_pre[(size_t)p * (ni + 1) + k] + cnt;
        }
      // node phases: partial sums over kBcrSub-node ranges of each instance
      // (the same alone or in a batch), task_sub ranges per task, about two
      // tasks per CTA or more
      bcr_npre.assign(ni + 1, 0);
      for (int k = 0; k < ni; ++k)
        bcr_npre[k + 1] = bcr_npre[k] + (int)((S->inst[k].nodes + kBcrSub - 1) / kBcrSub);
      pl.bcr.chunks = bcr_npre[ni];
      pl.bcr.rows = bcr_rows;
      pl.bcr.task_sub = (int)std::max<long long>(1, std::min<long long>(kBcrMaxTaskSub, pl.bcr.chunks / (2ll * bcr_nb)));
      bcr_tpre.assign(ni + 1, 0);
      for (int k = 0; k < ni; ++k)
        bcr_tpre[k + 1] = bcr_tpre[k] + (bcr_npre[k + 1] - bcr_npre[k] + pl.bcr.task_sub - 1) / pl.bcr.task_sub;
      pl.bcr.n_inst = ni;
      pl.bcr.phases = phases;
      pl.bcr.nd_wrows = nd_w;
      // dataflow sweeps when every instance is solved by nested dissection
      // (APIC_ND_FLOW=0: one grid barrier per tree level instead): a task
      // waits only for the fronts it reads (forward: its fronts' children,
      // backward: their parents), every front counting its finished tasks
      bool all_nd = true;
      for (int k = 0; k < ni; ++k) all_nd = all_nd && use_nd[k];
      if (const char* e = std::getenv("APIC_ND_FLOW")) all_nd = all_nd && std::atoi(e) != 0;
      pl.bcr.nd_flow = all_nd ? 1 : 0;
      nd_flow.clear();
      nd_need.clear();
      if (all_nd) {
        const int nf = (int)ndu.fronts.size();
        nd_need.assign(2 * (size_t)nf, 0);
        std::vector<std::pair<std::pair<int, int>, int2>> fe, be;  // ((key, instance), (task, instance))
        for (int k = 0; k < ni; ++k) {
          const BcrInst& B = bcr_in[k];
          for (int l = 0; l <= B.nd_depth; ++l) {
            for (int t = B.nd_ft[l]; t < B.nd_ft[l + 1]; ++t) fe.push_back({{B.nd_depth - l, k}, make_int2(t, k)});
            for (int t = B.nd_bt[l]; t < B.nd_bt[l + 1]; ++t) be.push_back({{l, k}, make_int2(t, k)});
          }
        }
        auto by_key = [](const std::pair<std::pair<int, int>, int2>& a, const std::pair<std::pair<int, int>, int2>& b) {
          return a.first < b.first || (a.first == b.first && a.second.x < b.second.x);
        };
        std::stable_sort(fe.begin(), fe.end(), by_key);
        std::stable_sort(be.begin(), be.end(), by_key);
        for (int sw = 0; sw < 2; ++sw)
          for (const auto& x : sw == 0 ? fe : be) {
            nd_flow.push_back(x.second);
            const NdTask& T = ndu.tasks[x.second.x];
            if (T.warp == 0) nd_need[(size_t)sw * nf + T.front] += 1;
            else
              for (int q = 0; q < T.n; ++q) nd_need[(size_t)sw * nf + T.front + q] += 1;
          }
        pl.bcr.nd_nf = (int)fe.size();
        pl.bcr.nd_nb = (int)be.size();
        pl.bcr.nd_fronts = nf;
      }
    } else {
      pl.bcr.n_inst = 0;
    }
  }
  const bool use_mg = pl.bcr.n_inst == 0;  // the multigrid hierarchy is only set up when it is used

  // ---- device memory ----
  DevPtrs& d = S->d;
  d.n_inst = ni;
  d.n_pop = S->n_pop;
  d.total_nodes = total_nodes;
  d.level_nodes = level_nodes;
  const size_t R = sizeof(Real);
  auto A = [&](size_t bytes) { return S->dalloc(bytes); };
  d.inst = (const Inst*)A(sizeof(Inst) * ni);
  d.pop = (const Pop*)A(sizeof(Pop) * S->n_pop);
  d.ps = (PopState*)A(sizeof(PopState) * S->n_pop);
  d.sol = (SolverState*)A(sizeof(SolverState) * ni);
  d.stp = (StepState*)A(sizeof(StepState) * ni);
  d.err = (int32_t*)A(sizeof(int32_t) * 4);
  d.cnt = (long long*)A(sizeof(long long) * 8);
  d.x1 = A(R * slots);
  d.x2 = A(R * slots);
  d.vR = A(R * slots);
  d.vZ = A(R * slots);
  d.vT = A(R * slots);
  d.holes = (int32_t*)A(sizeof(int32_t) * slots);
  d.total_cells = total_cells;
  for (const apic_config_t& c : S->cfg)
    if (c.sort_interval > 0) S->sort_interval = S->sort_interval ? std::min(S->sort_interval, c.sort_interval) : c.sort_interval;
  if (S->sort_interval > 0) {
    d.y1 = A(R * slots);
    d.y2 = A(R * slots);
    d.yR = A(R * slots);
    d.yZ = A(R * slots);
    d.yT = A(R * slots);
    d.cell_cnt = (unsigned*)A(sizeof(unsigned) * total_cells);
    d.cell_off = (unsigned long long*)A(sizeof(unsigned long long) * (total_cells + 1));
    d.scan_tmp = (unsigned long long*)A(sizeof(unsigned long long) * ((total_cells + 1023) / 1024 + 1));
  }
  double** node_arrays[] = {&d.rho, &d.phi, &d.phi_prev, &d.V, &d.Vinv, &d.bbc, &d.rscale, &d.b, &d.r, &d.rh, &d.p, &d.v, &d.s, &d.t, &d.ph, &d.sh};
  for (double** a : node_arrays) *a = (double*)A(sizeof(double) * total_nodes);
  for (const Inst& I : S->inst) S->floating = S->floating || (I.flags & APIC_FLOATING) != 0;
  if (S->floating) {
    d.bbc_g = (double*)A(sizeof(double) * total_nodes);
    d.phi_vac = (double*)A(sizeof(double) * total_nodes);
  }
  for (int k = 0; k < ni; ++k)
    if (S->inst[k].flags & APIC_BOLTZMANN) {
      S->boltz = true;
      S->newton = std::max(S->newton, S->cfg[k].newton_iters > 0 ? S->cfg[k].newton_iters : 8);
    }
  if (S->boltz) d.diag0 = (double*)A(sizeof(double) * total_nodes);
  if (const char* ne = std::getenv("APIC_NEWTON_ETA")) S->newton_eta = std::min(0.5, std::max(0.0, std::atof(ne)));
  S->phi_save = (double*)A(sizeof(double) * total_nodes);
  d.st64 = (double*)A(sizeof(double) * kSt * total_nodes);
  d.acc = (unsigned long long*)A(sizeof(unsigned long long) * 2 * total_nodes);
  d.G = A(2 * R * total_nodes);
  d.H = R == sizeof(float) ? (float*)A(4 * sizeof(float) * total_nodes) : nullptr;
  d.st = A(R * kSt * level_nodes);
  d.e = A(R * level_nodes);
  d.f = A(R * level_nodes);
  d.cinv = A(R * std::max<long long>(1, cinv_total));
  d.fac = A(R * std::max<long long>(1, fac_total));
  d.tab = (double*)A(sizeof(double) * tab_total);
  d.guide = (int32_t*)A(sizeof(int32_t) * tab_total);
  d.sgeo = (double*)A(sizeof(double) * 4 * en_total);
  d.tfix = (unsigned long long*)A(sizeof(unsigned long long) * std::max<long long>(1, bins_total));
  d.hist = (double*)A(sizeof(double) * hist_total);
  d.en = (double*)A(sizeof(double) * en_total);
  d.red = (double*)A(sizeof(double) * ni * kNRed * kRedBlocks);
  d.cred = (double*)A(sizeof(double) * ni * kNRed * kCoopMaxBlocks);
  d.bar = (unsigned*)A(sizeof(unsigned) * 4);
  d.wait_ns = kWaitNs;
  if (pl.bcr.n_inst > 0) {
    // blocks and tail inverses of every instance in one range (one L2
    // access-policy window covers them)
    d.bcr = (float*)A((size_t)pl.bcr.bytes);
    S->bcr_bytes = (size_t)pl.bcr.bytes;
    d.bcr_f = (float*)A(sizeof(float) * kBcrMaxRhs * (size_t)bcr_rows);  // up to kBcrMaxRhs right-hand sides
    d.bcr_e = (float*)A(sizeof(float) * kBcrMaxRhs * (size_t)bcr_rows);
    d.bcr_inst = (const BcrInst*)A(sizeof(BcrInst) * ni);
    d.bcr_kind = (const int32_t*)A(sizeof(int32_t) * bcr_kind.size());
    d.bcr_pre = (const int32_t*)A(sizeof(int32_t) * bcr_pre.size());
    d.bcr_npre = (const int32_t*)A(sizeof(int32_t) * bcr_npre.size());
    d.bcr_tpre = (const int32_t*)A(sizeof(int32_t) * bcr_tpre.size());
    d.bcr_part = (double*)A(sizeof(double) * (1 + kBcrMaxRhs) * (size_t)pl.bcr.chunks);
    if (!ndu.fronts.empty()) {
      d.nd_front = (const NdFront*)A(sizeof(NdFront) * ndu.fronts.size());
      d.nd_idx = (const int32_t*)A(sizeof(int32_t) * ndu.idx.size());
      d.nd_gather = (const int32_t*)A(sizeof(int32_t) * ndu.gather.size());
      d.nd_task = (const int4*)A(sizeof(NdTask) * ndu.tasks.size());
      d.nd_w = (float*)A(sizeof(float) * kBcrMaxRhs * (size_t)std::max<long long>(1, nd_w));
      if (pl.bcr.nd_flow) {
        d.nd_flow = (const int2*)A(sizeof(int2) * nd_flow.size());
        d.nd_need = (const int32_t*)A(sizeof(int32_t) * nd_need.size());
        d.nd_done = (unsigned*)A(sizeof(unsigned) * 2 * kBcrMaxRhs * (size_t)pl.bcr.nd_fronts);
      }
      if (S->status != APIC_OK) return S->status;
      if (pl.bcr.nd_flow) {
        S->h2d((int2*)d.nd_flow, nd_flow.data(), nd_flow.size());
        S->h2d((int32_t*)d.nd_need, nd_need.data(), nd_need.size());
      }
      S->h2d((NdFront*)d.nd_front, ndu.fronts.data(), ndu.fronts.size());
      S->h2d((int32_t*)d.nd_idx, ndu.idx.data(), ndu.idx.size());
      S->h2d((int32_t*)d.nd_gather, ndu.gather.data(), ndu.gather.size());
      S->h2d((NdTask*)d.nd_task, ndu.tasks.data(), ndu.tasks.size());
      {  // every task's matrix range (forward rows of FM, backward rows of NB)
        std::vector<longlong2> tr(ndu.tasks.size(), make_longlong2(0, 0));
        for (int k = 0; k < ni; ++k) {
          if (!use_nd[k]) continue;
          const BcrInst& B = bcr_in[k];
          for (int sw = 0; sw < 2; ++sw) {
            const int32_t* lv = sw == 0 ? B.nd_ft : B.nd_bt;
            for (int t = lv[0]; t < lv[B.nd_depth + 1]; ++t) {
              const NdTask& T = ndu.tasks[t];
              const NdFront& F0 = ndu.fronts[T.front];
              long long m0, m1;
              if (T.warp == 0) {
                const int width = sw == 0 ? F0.sp : F0.up;
                m0 = (sw == 0 ? F0.FM : F0.NB) + (long long)T.r0 * width;
                m1 = m0 + (sw == 0 || F0.u > 0 ? (long long)T.n * width : 0);
              } else {
                const NdFront& FL = ndu.fronts[T.front + T.n - 1];
                m0 = sw == 0 ? F0.FM : F0.NB;
                m1 = sw == 0 ? FL.FM + (long long)(FL.s + FL.u) * FL.sp : FL.NB + (long long)FL.s * FL.up;
              }
              tr[t] = make_longlong2(m0, m1);
            }
          }
        }
        d.nd_trange = (const longlong2*)A(sizeof(longlong2) * tr.size());
        if (S->status != APIC_OK) return S->status;
        S->h2d((longlong2*)d.nd_trange, tr.data(), tr.size());
        if (!S->sync()) return S->status;  // tr goes out of scope
      }
      for (int k = 0; k < ni; ++k) {
        if (!use_nd[k]) continue;
        const BcrInst& B = bcr_in[k];
        S->h2d(d.bcr + B.base, nds[k].fm.data(), nds[k].fm.size());
        S->h2d(d.bcr + B.base + nds[k].fm_total, nds[k].nb.data(), nds[k].nb.size());
      }
      if (!S->sync()) return S->status;  // the host copies are released below
      for (int k = 0; k < ni; ++k) nds[k] = NdFactor();
    }
    if (S->status != APIC_OK) return S->status;
    S->h2d((BcrInst*)d.bcr_inst, bcr_in.data(), bcr_in.size());
    S->h2d((int32_t*)d.bcr_kind, bcr_kind.data(), bcr_kind.size());
    S->h2d((int32_t*)d.bcr_pre, bcr_pre.data(), bcr_pre.size());
    S->h2d((int32_t*)d.bcr_npre, bcr_npre.data(), bcr_npre.size());
    S->h2d((int32_t*)d.bcr_tpre, bcr_tpre.data(), bcr_tpre.size());
    if (!S->sync()) return S->status;
    std::vector<float> blocks;
    std::vector<double> T, aug;
    for (int k = 0; k < ni; ++k) {
      const BcrInst& B = bcr_in[k];
      if (B.nd) continue;
      if (!bcr_factor(levels[k][0], B, blocks, T))
        return S->fail(APIC_ERR_INVALID_ARG, "block cyclic reduction: singular diagonal block");
      if (B.blocks > 0) S->h2d(d.bcr + B.base, blocks.data(), (size_t)(B.blocks * B.blk));
      // dense inverse of the tail system: Gauss-Jordan on the GPU (FP64), stored in FP32
      const int n = B.tail_n;
      double* work = (double*)S->dalloc(sizeof(double) * 2 * (size_t)n * n);
      double* fbuf = (double*)S->dalloc(sizeof(double) * ((size_t)n + 1));  // + the barrier counter
      float* dense = (float*)S->dalloc(sizeof(float) * (size_t)n * n);
      if (!work || !fbuf || !dense) return S->status;
      aug.assign((size_t)n * 2 * n, 0.0);
      for (int r = 0; r < n; ++r) {
        std::memcpy(aug.data() + (size_t)r * 2 * n, T.data() + (size_t)r * n, sizeof(double) * n);
        aug[(size_t)r * 2 * n + n + r] = 1.0;
      }
      S->h2d(work, aug.data(), aug.size());
      if (!S->ck(launch_dense_inverse<float>(work, fbuf, n, dense, (unsigned long long*)(fbuf + n), d.err, d.wait_ns,
                                             S->stream),
                 "dense inverse (tail)"))
        return S->status;
      // rows padded to 16 bytes (bulk copies of row chunks)
      if (!S->ck(cudaMemcpy2DAsync(d.bcr + B.tail, sizeof(float) * B.tail_np, dense, sizeof(float) * n,
                                   sizeof(float) * n, n, cudaMemcpyDeviceToDevice, S->stream),
                 "tail copy"))
        return S->status;
      // the host vectors are refilled for the next instance
      if (!S->sync() || !setup_wait_ok(S, "dense inverse (tail)")) return S->status;
      for (void* q : {(void*)dense, (void*)fbuf, (void*)work}) {
        auto it = std::find(S->blocks.begin(), S->blocks.end(), q);
        if (it != S->blocks.end()) S->blocks.erase(it);
        if (S->have_alloc) S->alloc.free(q, (void*)S->stream, S->alloc.ctx);
        else cudaFreeAsync(q, S->stream);
      }
    }
  }
  if (S->status != APIC_OK) return S->status;

  // ---- uploads ----
  S->h2d((Inst*)d.inst, S->inst.data(), ni);
  S->h2d((Pop*)d.pop, S->pop.data(), S->n_pop);
  std::vector<Real> tmp;
  for (int k = 0; k < ni; ++k) {
    const Inst& I = S->inst[k];
    S->h2d(d.tab + I.tab_off, tabs[k].data(), tabs[k].size());
    std::vector<int32_t> guide = guide_tables(tabs[k]);
    S->h2d(d.guide + I.tab_off, guide.data(), guide.size());
    std::vector<double> sgeo = surface_geometry(I);
    S->h2d(d.sgeo + 4 * I.en_off, sgeo.data(), sgeo.size());
    S->h2d(d.V + I.node_off, vols[k].data(), vols[k].size());
    std::vector<double> vinv(vols[k].size());
    for (size_t q = 0; q < vinv.size(); ++q) vinv[q] = 1.0 / vols[k][q];
    S->h2d(d.Vinv + I.node_off, vinv.data(), vinv.size());
    if (!S->sync()) return S->status;  // vinv goes out of scope
    S->h2d(d.rscale + I.node_off, rscs[k].data(), rscs[k].size());
    S->h2d(d.bbc + I.node_off, bbcs[k].data(), bbcs[k].size());
    S->h2d(d.st64 + (long long)kSt * I.node_off, levels[k][0].st.data(), levels[k][0].st.size());
    if (I.flags & APIC_BOLTZMANN)
      S->h2d(d.diag0 + I.node_off, levels[k][0].st.data() + (size_t)st_slot(0, 0) * I.nodes, (size_t)I.nodes);
    for (int l = 0; l < I.n_levels; ++l) {
      const HostLevel& H = levels[k][l];
      tmp.assign(H.st.begin(), H.st.end());
      S->h2d((Real*)d.st + I.lv[l].st, tmp.data(), tmp.size());
    }
    if (use_mg) {
      // Gauss-Jordan on the GPU: n x 2n FP64 workspace, result stored in the particle precision
      int nu = I.coarse_n;
      double* work = (double*)S->dalloc(sizeof(double) * 2 * (size_t)nu * nu);
      double* fbuf = (double*)S->dalloc(sizeof(double) * ((size_t)nu + 1));  // + the barrier counter
      if (!work || !fbuf) return S->status;
      std::vector<double> aug((size_t)nu * 2 * nu, 0.0);
      for (int r = 0; r < nu; ++r) {
        std::memcpy(aug.data() + (size_t)r * 2 * nu, cinvs[k].data() + (size_t)r * nu, sizeof(double) * nu);
        aug[(size_t)r * 2 * nu + nu + r] = 1.0;
      }
      S->h2d(work, aug.data(), aug.size());
      if (!S->ck(launch_dense_inverse<Real>(work, fbuf, nu, (Real*)d.cinv + I.cinv_off,
                                            (unsigned long long*)(fbuf + nu), d.err, d.wait_ns, S->stream),
                 "dense inverse"))
        return S->status;
      if (!S->sync() || !setup_wait_ok(S, "dense inverse")) return S->status;
      // release the workspace
      for (void* q : {(void*)fbuf, (void*)work}) {
        auto it = std::find(S->blocks.begin(), S->blocks.end(), q);
        if (it != S->blocks.end()) S->blocks.erase(it);
        if (S->have_alloc) S->alloc.free(q, (void*)S->stream, S->alloc.ctx);
        else cudaFreeAsync(q, S->stream);
      }
    }
    // initial potential: the vacuum solution, linear in x1 (phi = 0 without field)
    std::vector<double> phi((size_t)I.nodes, 0.0);
    if (!(I.flags & APIC_NO_FIELD))
      for (int i = 0; i <= I.n1; ++i)
        for (int j = 0; j <= I.n2; ++j)
          phi[(size_t)i * I.N2 + j] = I.phi_g + (I.phi_out - I.phi_g) * (x1_node_h(I, i) + 1.0) / (I.x1_out + 1.0);
    S->h2d(d.phi + I.node_off, phi.data(), phi.size());
    // tables are synchronous inputs of host vectors: wait before they go out of scope
    if (!S->sync()) return S->status;
  }
  // line factorisations of every level (constant in time)
  for (int l = 0; l < kMaxLevels && use_mg; ++l) {
    int lines1 = 0, lines2 = 0, k1 = 1, k2 = 1;
    bool any = false;
    for (const Inst& I : S->inst) {
      if (l >= I.n_levels) continue;
      any = true;
      lines1 = std::max(lines1, I.lv[l].N2);
      lines2 = std::max(lines2, I.lv[l].N1);
      k1 = std::max(k1, (I.lv[l].n1 - 1 + 31) / 32);
      k2 = std::max(k2, (I.lv[l].n2 + 1 + 31) / 32);
    }
    if (!any) break;
    launch_line_factor<Real>(d, l, 0, lines1, k1, S->stream);
    launch_line_factor<Real>(d, l, 1, lines2, k2, S->stream);
  }
  if (!S->ck(cudaGetLastError(), "line factorisation")) return S->status;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  S->push_grid = std::max(1, sms) * 4;
  // APIC_COND_LOOP=0: the fixed, early-exiting Krylov loop instead of the
  // conditional while node (profilers do not replay kernels of graphs that
  // hold conditional nodes)
  if (const char* cl = std::getenv("APIC_COND_LOOP")) S->cond_loop = std::atoi(cl) != 0;
  for (const Inst& I : S->inst) {
    S->max_n2 = std::max(S->max_n2, I.n2);
    S->max_n1 = std::max(S->max_n1, I.n1);
  }
  push_window_rows<Real>(S->max_n2);  // the occupancy queries happen here, not inside a graph capture
  sort_setup<Real>(S->max_n1);
  for (const Inst& I : S->inst) S->chord = S->chord || (I.flags & APIC_CHORD_ABSORB) != 0;
  // the whole Poisson solve as one cooperative kernel, unless disabled or not co-residable
  const char* env = std::getenv("APIC_SOLVER");
  // one cooperative launch per solve for a single instance; batches use the
  // per-phase kernels, whose grids span every instance at once
  bool want_coop = ni == 1;
  if (env && std::string(env) == "kernels") want_coop = false;
  if (env && std::string(env) == "coop") want_coop = ni <= kCoopMaxInst;
  S->coop = want_coop ? coop_blocks<Real>(S->plan, sms) : 0;
  if (const char* nbv = std::getenv("APIC_COOP_BLOCKS")) S->coop = std::min(S->coop, std::max(1, std::atoi(nbv)));
  if (pl.bcr.n_inst > 0) S->coop = bcr_nb;
  // Optionally (APIC_L2_PERSIST=1) keep the reduction's blocks in L2 across
  // steps: a persisting access window on the solve's graph node, with this
  // context's L2 set-aside (released with the context).  Off by default: on
  // the bench the set-aside slowed the push and injection by more than it
  // saved in the solve.
  if (pl.bcr.n_inst > 0 && std::getenv("APIC_L2_PERSIST") && std::string(std::getenv("APIC_L2_PERSIST")) == "1") {
    int maxp = 0, maxw = 0;
    cudaDeviceGetAttribute(&maxp, cudaDevAttrMaxPersistingL2CacheSize, dev);
    cudaDeviceGetAttribute(&maxw, cudaDevAttrMaxAccessPolicyWindowSize, dev);
    size_t want = std::min<size_t>(S->bcr_bytes, (size_t)std::max(0, maxp));
    if (want > 0 && maxw > 0 && cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, want) == cudaSuccess)
      S->l2_persist = want;
    cudaGetLastError();
  }
  cudaGetLastError();
  if (S->floating && !vacuum_fields<Real>(S)) return S->status;
  return S->sync() ? APIC_OK : S->status;
}

extern "C" int apic_create_batch(const apic_config_t* cfgs, int32_t n, void* stream,
                                 const apic_allocator_t* allocator, apic_sim** out) {
  if (!out) return APIC_ERR_INVALID_ARG;
  *out = nullptr;
  if (!cfgs || n < 1) return APIC_ERR_INVALID_ARG;
  std::string why;
  for (int k = 0; k < n; ++k) {
    int rc = validate(cfgs[k], why);
    if (rc != APIC_OK) {
      std::fprintf(stderr, "apic_create: instance %d: %s\n", k, why.c_str());
      return rc;
    }
    if (cfgs[k].precision != cfgs[0].precision) return APIC_ERR_INVALID_ARG;
  }
  apic_sim* S = new apic_sim();
  S->precision = cfgs[0].precision;
  S->n_inst = n;
  S->cfg.assign(cfgs, cfgs + n);
  S->stream = (cudaStream_t)stream;
  if (allocator && allocator->alloc && allocator->free) {
    S->alloc = *allocator;
    S->have_alloc = true;
  }
  if (!S->ck(cudaStreamCreateWithFlags(&S->cap, cudaStreamNonBlocking), "cudaStreamCreate") ||
      !S->ck(cudaStreamCreateWithFlags(&S->cap2, cudaStreamNonBlocking), "cudaStreamCreate") ||
      !S->ck(cudaMallocHost(&S->h_err, 16), "cudaMallocHost")) {
    int rc = S->status;
    apic_destroy(S);
    return rc;
  }
  int rc = S->precision == APIC_FP64 ? setup<double>(S) : setup<float>(S);
  if (rc != APIC_OK) {
    std::fprintf(stderr, "apic_create: %s\n", S->msg.c_str());
    apic_destroy(S);
    return rc;
  }
  *out = S;
  return APIC_OK;
}

extern "C" int apic_create(const apic_config_t* cfg, void* stream, const apic_allocator_t* allocator, apic_sim** out) {
  return apic_create_batch(cfg, 1, stream, allocator, out);
}

// Drop the captured step graphs (the next step captures them again).
static void drop_graphs(apic_sim* S) {
  for (int q = 0; q < 2; ++q) {
    if (S->exec[q]) cudaGraphExecDestroy(S->exec[q]);
    if (S->graph[q]) cudaGraphDestroy(S->graph[q]);
    if (S->sort_exec[q]) cudaGraphExecDestroy(S->sort_exec[q]);
    if (S->sort_graph[q]) cudaGraphDestroy(S->sort_graph[q]);
    S->exec[q] = nullptr;
    S->graph[q] = nullptr;
    S->sort_exec[q] = nullptr;
    S->sort_graph[q] = nullptr;
    for (int p = 0; p < APIC_NPHASE; ++p) {
      if (S->phase_exec[q][p]) cudaGraphExecDestroy(S->phase_exec[q][p]);
      if (S->phase_graph[q][p]) cudaGraphDestroy(S->phase_graph[q][p]);
      S->phase_exec[q][p] = nullptr;
      S->phase_graph[q][p] = nullptr;
    }
  }
}

extern "C" int apic_destroy(apic_sim* S) {
  if (!S) return APIC_OK;
  if (S->stream || S->cap) cudaStreamSynchronize(S->stream);
  drop_graphs(S);
  for (int p = 0; p <= APIC_NPHASE; ++p)
    if (S->ev[p]) cudaEventDestroy(S->ev[p]);
  for (cudaEvent_t e : S->sort_ev)
    if (e) cudaEventDestroy(e);
  S->dfree_all();
  cudaStreamSynchronize(S->stream);
  if (S->cap) cudaStreamDestroy(S->cap);
  if (S->cap2) cudaStreamDestroy(S->cap2);
  if (S->h_err) cudaFreeHost(S->h_err);
  if (S->h_tally) cudaFreeHost(S->h_tally);
  delete S;
  return APIC_OK;
}

// ---------------------------------------------------------------------------
// Stepping.
// ---------------------------------------------------------------------------
template <class Real>
static void enqueue_solver_iterations_fixed(apic_sim* S, const DevPtrs& d, cudaStream_t s) {
  int most = 0;
  for (const Inst& I : S->inst) most = std::max(most, I.max_iter);
  for (int it = 0; it < most; ++it) {
    launch_bicg_iter<Real>(d, S->plan, s);
    launch_bicg_check(d, 0, 0, s);
  }
}

// Inside an open capture on stream s: a while-node whose body is one Krylov
// iteration followed by the test kernel that sets the loop condition.
template <class Real>
static bool enqueue_solver_loop(apic_sim* S, const DevPtrs& d, cudaStream_t s) {
  cudaStreamCaptureStatus st;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  if (cudaStreamGetCaptureInfo(s, &st, nullptr, &g, &deps, nullptr, &nd) != cudaSuccess) return false;
  cudaGraphConditionalHandle h;
  if (cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault) != cudaSuccess) return false;
  cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t cn;
  if (cudaGraphAddNode(&cn, g, deps, nullptr, nd, &cp) != cudaSuccess) return false;
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  if (cudaStreamUpdateCaptureDependencies(s, &cn, nullptr, 1, cudaStreamSetCaptureDependencies) != cudaSuccess)
    return false;
  if (cudaStreamBeginCaptureToGraph(S->cap2, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) !=
      cudaSuccess)
    return false;
  launch_bicg_iter<Real>(d, S->plan, S->cap2);
  launch_bicg_check(d, h, 1, S->cap2);
  cudaGraph_t tmp = nullptr;
  return cudaStreamEndCapture(S->cap2, &tmp) == cudaSuccess;
}

// One cooperative launch for the whole solve: block cyclic reduction when
// set up, else the multigrid-preconditioned BiCGSTAB.
template <class Real>
static cudaError_t solve_coop(apic_sim* S, const DevPtrs& d, cudaStream_t s, int bcr_mode = 0, int only = -1) {
  if (S->plan.bcr.n_inst > 0) return launch_solve_bcr(d, S->plan, S->coop, bcr_mode, only, s);
  return launch_solve_coop<Real>(d, S->plan, S->coop, s);
}

// Kernels of phase p of one step (deposit->rho, Poisson, fields, push, inject, bookkeeping).
template <class Real>
static bool enqueue_phase(apic_sim* S, const DevPtrs& d, int p, cudaStream_t s) {
  switch (p) {
    case 0:
      if (S->plan.bcr.n_inst == 0) launch_rho<Real>(d, s);  // the reduction solve forms rho itself
      break;
    case 1:
      // Boltzmann electrons: newton Newton iterations, each a linear solve
      for (int k = 0; k < (S->boltz ? S->newton : 1); ++k) {
        if (S->boltz) launch_newton(d, -1, k == S->newton - 1 ? 0.0 : S->newton_eta, s);
        if (S->coop > 0) {
          if (solve_coop<Real>(S, d, s, kBcrRho | kBcrFields) != cudaSuccess) return false;
          continue;
        }
        launch_bicg_init<Real>(d, s);
        if (S->cond_loop) {
          if (!enqueue_solver_loop<Real>(S, d, s)) return false;
        } else {
          enqueue_solver_iterations_fixed<Real>(S, d, s);
        }
      }
      if (S->boltz) launch_newton_end(d, s);
      break;
    case 2:
      if (S->plan.bcr.n_inst == 0) {  // the reduction solve ends with them
        launch_gradients<Real>(d, s);
        launch_surface(d, s);
      }
      if (S->floating) {  // the isolated grains' correction (chosen by the surface step), then the gradients again
        launch_float_phi(d, s);
        launch_gradients<Real>(d, s);
      }
      break;
    case 3:
      launch_push<Real>(d, S->push_grid, S->max_n2, S->chord, S->win_rows, S->chunk_group, S->chunk_items, S->slots, s);
      break;
    case 4: launch_inject<Real>(d, S->max_inj, s); break;
    case 5: launch_step_end(d, s); break;
    case 6: launch_sort<Real>(d, S->push_grid, S->max_n1, s); break;  // not a step phase: the particle sort
  }
  return true;
}

// Persisting L2 window over the reduction blocks on the solve's kernel node.
static void set_persisting_window(apic_sim* S, const DevPtrs& d, cudaGraph_t g) {
  if (S->l2_persist == 0 || !d.bcr) return;
  size_t n = 0;
  if (cudaGraphGetNodes(g, nullptr, &n) != cudaSuccess || n == 0) return;
  std::vector<cudaGraphNode_t> nodes(n);
  if (cudaGraphGetNodes(g, nodes.data(), &n) != cudaSuccess) return;
  int dev = 0, maxw = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&maxw, cudaDevAttrMaxAccessPolicyWindowSize, dev);
  for (cudaGraphNode_t node : nodes) {
    cudaGraphNodeType t;
    if (cudaGraphNodeGetType(node, &t) != cudaSuccess || t != cudaGraphNodeTypeKernel) continue;
    cudaKernelNodeParams kp;
    if (cudaGraphKernelNodeGetParams(node, &kp) != cudaSuccess || kp.func != bcr_kernel(S->plan)) continue;
    cudaKernelNodeAttrValue v;
    std::memset(&v, 0, sizeof(v));
    v.accessPolicyWindow.base_ptr = (void*)d.bcr;
    v.accessPolicyWindow.num_bytes = std::min<size_t>(S->bcr_bytes, (size_t)maxw);
    v.accessPolicyWindow.hitRatio =
        (float)std::min(1.0, (double)S->l2_persist / (double)v.accessPolicyWindow.num_bytes);
    v.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
    v.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
    cudaGraphKernelNodeSetAttribute(node, cudaKernelNodeAttributeAccessPolicyWindow, &v);
  }
  cudaGetLastError();
}

// Capture phases [p0, p1) into one executable graph.  If the while-node cannot
// be built, the capture is redone once with a fixed, early-exiting loop.
template <class Real>
static bool capture(apic_sim* S, const DevPtrs& d, int p0, int p1, cudaGraph_t* graph, cudaGraphExec_t* exec) {
  for (int attempt = 0; attempt < 2; ++attempt) {
    cudaStream_t s = S->cap;
    if (!S->ck(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal), "begin capture")) return false;
    bool ok = true;
    for (int p = p0; p < p1 && ok; ++p) ok = enqueue_phase<Real>(S, d, p, s);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(s, &g);
    if (ok && e == cudaSuccess) {
      *graph = g;
      set_persisting_window(S, d, g);
      return S->ck(cudaGraphInstantiate(exec, g, 0), "graph instantiate");
    }
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    if (!S->cond_loop) return S->ck(e == cudaSuccess ? cudaErrorUnknown : e, "step capture");
    S->cond_loop = false;  // retry without the conditional node
  }
  return false;
}

static int read_status(apic_sim* S);

extern "C" int apic_check_wait_limit(apic_sim* S, int64_t limit_ns) {
  if (!S) return APIC_ERR_INVALID_ARG;
  if (limit_ns < 1000 || limit_ns > 10000000000ll) return S->fail(APIC_ERR_INVALID_ARG, "limit_ns out of range");
  if (S->status != APIC_OK) return S->status;
  DevPtrs w = S->d;
  w.bar = (unsigned*)S->dalloc(256);  // a zeroed barrier counter of its own
  if (!w.bar) return S->status;
  w.wait_ns = (unsigned long long)limit_ns;
  launch_wait_check(w, 4, S->stream);
  if (!S->ck(cudaGetLastError(), "wait check launch")) return S->status;
  return read_status(S);
}

static int read_status(apic_sim* S) {
  if (!S->d2h(S->h_err, S->d.err, 1) || !S->sync()) return S->status;
  int e = S->h_err[0];
  if (e & kErrCapacity) return S->fail(APIC_ERR_CAPACITY, "particle capacity exceeded");
  if (e & kErrNonFinite) return S->fail(APIC_ERR_NONFINITE, "non-finite field or residual");
  if (e & kErrNotConverged) return S->fail(APIC_ERR_NOT_CONVERGED, "Poisson iteration limit reached");
  if (e & kErrTimeout) return S->fail(APIC_ERR_TIMEOUT, "grid barrier of the cooperative solver timed out");
  return APIC_OK;
}

template <class Real>
static bool redeposit(apic_sim* S) {
  if (!S->dirty) return true;
  if (!S->ck(cudaMemsetAsync(S->d.acc, 0, sizeof(unsigned long long) * 2 * S->d.total_nodes, S->stream), "memset"))
    return false;
  launch_deposit_all<Real>(S->view(S->par), S->push_grid, S->max_n2, S->stream);
  S->dirty = false;
  return true;
}

template <class Real>
static bool ensure_graphs(apic_sim* S) {
  if (S->exec[0]) return true;
  if (!S->sync()) return false;
  int npar = S->sort_interval > 0 ? 2 : 1;
  for (int p = 0; p < npar; ++p) {
    DevPtrs v = S->view(p);
    if (!capture<Real>(S, v, 0, APIC_NPHASE, &S->graph[p], &S->exec[p])) return false;
    if (S->sort_interval > 0 && !capture<Real>(S, v, 6, 7, &S->sort_graph[p], &S->sort_exec[p])) return false;
  }
  return true;
}

// Sort (when due) and swap the particle buffers; then one step graph.
template <class Real>
static bool launch_step(apic_sim* S, cudaGraphExec_t const* step_exec) {
  if (S->sort_interval > 0 && S->host_step % S->sort_interval == 0) {
    if (!S->ck(cudaGraphLaunch(S->sort_exec[S->par], S->stream), "sort launch")) return false;
    S->par ^= 1;
    S->sorts += 1;
  }
  if (step_exec && !S->ck(cudaGraphLaunch(step_exec[S->par], S->stream), "graph launch")) return false;
  S->host_step += 1;
  return true;
}

template <class Real>
static int step_impl(apic_sim* S, int n) {
  if (!redeposit<Real>(S) || !ensure_graphs<Real>(S)) return S->status;
  for (int k = 0; k < n; ++k)
    if (!launch_step<Real>(S, S->exec)) return S->status;
  if (!S->ck(cudaGetLastError(), "launch")) return S->status;
  return read_status(S);
}

template <class Real>
static int step_timed_impl(apic_sim* S, int n) {
  if (!redeposit<Real>(S) || !ensure_graphs<Real>(S)) return S->status;
  if (!S->phase_exec[0][0]) {
    if (!S->sync()) return S->status;
    int npar = S->sort_interval > 0 ? 2 : 1;
    for (int q = 0; q < npar; ++q)
      for (int p = 0; p < APIC_NPHASE; ++p)
        if (!capture<Real>(S, S->view(q), p, p + 1, &S->phase_graph[q][p], &S->phase_exec[q][p])) return S->status;
    for (int p = 0; p <= APIC_NPHASE; ++p)
      if (!S->ev[p] && !S->ck(cudaEventCreate(&S->ev[p]), "event create")) return S->status;
    for (cudaEvent_t& e : S->sort_ev)
      if (!e && !S->ck(cudaEventCreate(&e), "event create")) return S->status;
  }
  for (int k = 0; k < n; ++k) {
    // the sort when due, timed on its own
    const bool sorting = S->sort_interval > 0 && S->host_step % S->sort_interval == 0;
    if (sorting) S->ck(cudaEventRecord(S->sort_ev[0], S->stream), "event record");
    if (!launch_step<Real>(S, nullptr)) return S->status;
    if (sorting) S->ck(cudaEventRecord(S->sort_ev[1], S->stream), "event record");
    S->host_step -= 1;
    S->ck(cudaEventRecord(S->ev[0], S->stream), "event record");
    for (int p = 0; p < APIC_NPHASE; ++p) {
      if (!S->ck(cudaGraphLaunch(S->phase_exec[S->par][p], S->stream), "graph launch")) return S->status;
      S->ck(cudaEventRecord(S->ev[p + 1], S->stream), "event record");
    }
    S->host_step += 1;
    if (!S->ck(cudaEventSynchronize(S->ev[APIC_NPHASE]), "event sync")) return S->status;
    for (int p = 0; p < APIC_NPHASE; ++p) {
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, S->ev[p], S->ev[p + 1]);
      S->phase_ms[p] += ms;
    }
    if (sorting) {
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, S->sort_ev[0], S->sort_ev[1]);
      S->sort_ms += ms;
      S->timed_sorts += 1;
    }
  }
  S->timed_steps += n;
  return read_status(S);
}

extern "C" int apic_step_timed(apic_sim* S, int32_t n_steps) {
  if (!S) return APIC_ERR_INVALID_ARG;
  if (S->status != APIC_OK) return S->status;
  if (n_steps < 0) return APIC_ERR_INVALID_ARG;
  if (n_steps == 0) return APIC_OK;
  return S->precision == APIC_FP64 ? step_timed_impl<double>(S, n_steps) : step_timed_impl<float>(S, n_steps);
}

// The vector push's default chunk (launch_push): 32 particles per thread when
// the batch's slots give every CTA two dozen 8192-particle chunks.
static int push4_default_items(const apic_sim* S) {
  const int grid = std::max(1, S->push_grid / 4 * (int)APIC_PUSH4_MIN_BLOCKS);
  return S->slots >= 24ll * 8192 * grid ? 32 : 16;
}

extern "C" int apic_stats(apic_sim* S, apic_stats_t* out) {
  if (!S || !out) return APIC_ERR_INVALID_ARG;
  long long cnt = 0;
  StepState stp;
  if (!S->sync() || !S->d2h(&cnt, S->d.cnt, 1) || !S->d2h(&stp, S->d.stp, 1) || !S->sync()) return S->status;
  std::memset(out, 0, sizeof(*out));
  out->steps = stp.step;
  out->poisson_loop_iters = cnt;
  int vcycle = S->plan.max_tail * 10 + 1;
  int most = 0;
  for (const Inst& I : S->inst) most = std::max(most, I.max_iter);
  if (S->plan.bcr.n_inst > 0) {
    out->kernels_per_iter = 0;   // solve, density and fields in one cooperative launch
    out->kernels_per_step = 4;   // + push, injection, bookkeeping
  } else if (S->coop > 0) {
    out->kernels_per_iter = 0;   // the whole solve is one cooperative launch
    out->kernels_per_step = S->boltz ? 7 + 2 * S->newton : 7;  // per Newton iteration: linearisation + solve
  } else if (S->boltz) {  // per Newton iteration: linearisation and BiCGSTAB set-up; then the diagonal back
    out->kernels_per_iter = 6 + 2 * vcycle;
    out->kernels_per_step = 6 + 1 + S->newton * (2 + (S->cond_loop ? 0 : most * out->kernels_per_iter));
  } else {
    out->kernels_per_iter = 6 + 2 * vcycle;
    out->kernels_per_step = 7 + (S->cond_loop ? 0 : most * out->kernels_per_iter);
  }
  if (S->floating) out->kernels_per_step += 2;  // the isolated grains' correction and the gradients again
  out->timed_steps = S->timed_steps;
  out->sort_interval = S->sort_interval;
  out->win_rows = S->win_rows > 0 ? S->win_rows
                                  : (S->precision == APIC_FP64 ? push_window_rows<double>(S->max_n2)
                                                               : push_window_rows<float>(S->max_n2));
  out->chunk_group = S->chunk_group > 0 ? S->chunk_group : 4;
  out->chunk_items = S->precision == APIC_FP64 ? 0 : (S->chunk_items > 0 ? S->chunk_items : push4_default_items(S));
  out->solver = S->plan.bcr.n_inst > 0 ? (S->d.nd_front ? APIC_SOLVER_ND : APIC_SOLVER_BCR)
                                       : (S->coop > 0 ? APIC_SOLVER_MG_COOP : APIC_SOLVER_MG_KERNELS);
  out->sorts = S->sorts;
  out->kernels_per_sort = 6;
  out->timed_sorts = S->timed_sorts;
  out->sort_ms = S->sort_ms;
  for (int p = 0; p < APIC_NPHASE; ++p) out->phase_ms[p] = S->phase_ms[p];
  return APIC_OK;
}

// Autotuning: `trial` steps (whole sort intervals) with each candidate sort
// interval (each trial starts with a sort), CUDA events on the simulation's
// stream, the fastest interval kept; then at that interval the push's chunk
// group and deposit-window rows, one warm-up interval and the timed steps per
// candidate with the step graphs recaptured.
static const int kTuneIntervals[APIC_TUNE_CANDIDATES] = {2, 4, 6, 8, 12, 16, 24};

template <class Real>
static int autotune_impl(apic_sim* S, int trial, int32_t* chosen, double* ms_out) {
  if (!redeposit<Real>(S) || !ensure_graphs<Real>(S)) return S->status;
  if (S->sort_interval <= 0) {  // sorting is off (no second particle buffer)
    *chosen = 0;
    return APIC_OK;
  }
  cudaEvent_t a = nullptr, b = nullptr;
  if (!S->ck(cudaEventCreate(&a), "event") || !S->ck(cudaEventCreate(&b), "event")) return S->status;
  double best = 1e300;
  int best_c = S->sort_interval;
  for (int q = 0; q < APIC_TUNE_CANDIDATES && S->status == APIC_OK; ++q) {
    const int c = kTuneIntervals[q];
    // whole sort intervals: a trial shorter than the interval would time only
    // the freshly sorted steps and favour long intervals
    const int n = c * ((trial + c - 1) / c);
    S->ck(cudaEventRecord(a, S->stream), "event record");
    for (int k = 0; k < n; ++k) {
      if (k % c == 0) {
        if (!S->ck(cudaGraphLaunch(S->sort_exec[S->par], S->stream), "sort launch")) break;
        S->par ^= 1;
        S->sorts += 1;
      }
      if (!S->ck(cudaGraphLaunch(S->exec[S->par], S->stream), "graph launch")) break;
      S->host_step += 1;
    }
    S->ck(cudaEventRecord(b, S->stream), "event record");
    if (!S->ck(cudaEventSynchronize(b), "event sync")) break;
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, a, b);
    const double per = (double)ms / n;
    if (ms_out) ms_out[q] = per;
    if (per < best) {
      best = per;
      best_c = c;
    }
  }
  if (S->status != APIC_OK) {
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return S->status;
  }
  S->sort_interval = best_c;
  *chosen = best_c;
  // the push's tiles at that interval: chunks per group, then deposit-window
  // rows; each candidate recaptures the step graphs and runs whole intervals
  auto time_steps = [&]() -> double {
    if (!S->sync() || !ensure_graphs<Real>(S)) return 1e300;
    const int n = best_c * ((trial + best_c - 1) / best_c);
    for (int k = 0; k < best_c && S->status == APIC_OK; ++k) launch_step<Real>(S, S->exec);  // warm-up interval
    S->ck(cudaEventRecord(a, S->stream), "event record");
    for (int k = 0; k < n && S->status == APIC_OK; ++k) launch_step<Real>(S, S->exec);
    S->ck(cudaEventRecord(b, S->stream), "event record");
    if (!S->ck(cudaEventSynchronize(b), "event sync")) return 1e300;
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, a, b);
    return (double)ms / n;
  };
  const int groups[] = {2, 4, 8};
  double best_t = 1e300;
  int best_g = S->chunk_group, best_r = S->win_rows;
  for (int g : groups) {
    S->chunk_group = g;
    drop_graphs(S);
    const double t = time_steps();
    if (t < best_t) {
      best_t = t;
      best_g = g;
    }
  }
  S->chunk_group = best_g;
  const int rows_cand[] = {2, 4, 6, 8, 12, 16};
  for (int r : rows_cand) {
    S->win_rows = r;
    drop_graphs(S);
    const double t = time_steps();
    if (t < best_t) {
      best_t = t;
      best_r = r;
    }
  }
  S->win_rows = best_r;
  int best_i = S->chunk_items;
  if (S->precision != APIC_FP64) {  // the vector push's chunk size
    const int items_cand[] = {16, 32};
    for (int c : items_cand) {
      S->chunk_items = c;
      drop_graphs(S);
      const double t = time_steps();
      if (t < best_t) {
        best_t = t;
        best_i = c;
      }
    }
  }
  S->chunk_items = best_i;
  drop_graphs(S);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (S->status != APIC_OK) return S->status;
  return read_status(S);
}

extern "C" int apic_autotune(apic_sim* S, int32_t steps_per_trial, int32_t* sort_interval, double* ms_per_step) {
  if (!S || !sort_interval || steps_per_trial < 1) return APIC_ERR_INVALID_ARG;
  if (S->status != APIC_OK) return S->status;
  return S->precision == APIC_FP64 ? autotune_impl<double>(S, steps_per_trial, sort_interval, ms_per_step)
                                   : autotune_impl<float>(S, steps_per_trial, sort_interval, ms_per_step);
}

extern "C" int apic_set_schedule(apic_sim* S, int32_t sort_interval, int32_t win_rows, int32_t chunk_group,
                                 int32_t chunk_items) {
  if (!S) return APIC_ERR_INVALID_ARG;
  if (S->status != APIC_OK) return S->status;
  if (sort_interval < 0 || (sort_interval > 0 && S->sort_interval <= 0)) return APIC_ERR_INVALID_ARG;
  if (win_rows != 0 && (win_rows < 2 || win_rows > 16)) return APIC_ERR_INVALID_ARG;
  if (chunk_group < 0 || chunk_group > 64) return APIC_ERR_INVALID_ARG;
  if (chunk_items != 0 && chunk_items != 16 && chunk_items != 32) return APIC_ERR_INVALID_ARG;
  if (!S->sync()) return S->status;
  if (sort_interval > 0) S->sort_interval = sort_interval;
  if (win_rows > 0) S->win_rows = win_rows;
  if (chunk_group > 0) S->chunk_group = chunk_group;
  if (chunk_items > 0 && S->precision != APIC_FP64) S->chunk_items = chunk_items;
  drop_graphs(S);  // recaptured at the next step
  return APIC_OK;
}

extern "C" int apic_step(apic_sim* S, int32_t n_steps) {
  if (!S) return APIC_ERR_INVALID_ARG;
  if (S->status != APIC_OK) return S->status;
  if (n_steps < 0) return APIC_ERR_INVALID_ARG;
  if (n_steps == 0) return APIC_OK;
  return S->precision == APIC_FP64 ? step_impl<double>(S, n_steps) : step_impl<float>(S, n_steps);
}

// ---------------------------------------------------------------------------
// Injection.
// ---------------------------------------------------------------------------
template <class Real>
static int inject_impl(apic_sim* S, int inst, int species, long long n, int mode, const double* st) {
  int pop = S->inst[inst].pop0 + species;
  const Pop& P = S->pop[pop];
  PopState ps;
  if (!S->sync() || !S->d2h(&ps, S->d.ps + pop, 1) || !S->sync()) return S->status;
  if (mode == APIC_FLUX_SURFACE) {
    if (ps.n + n > P.cap) return APIC_ERR_CAPACITY;
    ps.n_inj = n;
    ps.inj_stored = 0;
    if (!S->h2d(S->d.ps + pop, &ps, 1)) return S->status;
    launch_inject<Real>(S->view(S->par), n, S->stream);
    launch_finish_injection(S->d, pop, S->stream);
    S->dirty = true;
    return read_status(S);
  }
  if (ps.n + n > P.cap) return APIC_ERR_CAPACITY;
  if (mode == APIC_LOAD_VOLUME) {
    launch_load<Real>(S->view(S->par), pop, ps.n, n, ps.draws, 1, S->stream);
    ps.draws += n;
  } else {
    double* tmp = (double*)S->dalloc(sizeof(double) * 5 * (size_t)n);
    if (!tmp) return S->status;
    if (!S->h2d(tmp, st, 5 * (size_t)n)) return S->status;
    launch_explicit<Real>(S->view(S->par), pop, ps.n, n, tmp, S->stream);
    if (!S->sync()) return S->status;
    // release the staging buffer now
    S->blocks.pop_back();
    if (S->have_alloc) S->alloc.free(tmp, (void*)S->stream, S->alloc.ctx);
    else cudaFreeAsync(tmp, S->stream);
  }
  ps.n += n;
  ps.loaded += n;
  if (!S->h2d(S->d.ps + pop, &ps, 1) || !S->sync()) return S->status;
  S->dirty = true;
  return S->ck(cudaGetLastError(), "inject") ? APIC_OK : S->status;
}

extern "C" int apic_inject(apic_sim* S, int32_t instance, int32_t species, int64_t n, int32_t mode,
                           const double* explicit_state) {
  if (!S) return APIC_ERR_INVALID_ARG;
  if (S->status != APIC_OK) return S->status;
  if (instance < 0 || instance >= S->n_inst || species < 0 || species >= S->inst[instance].n_species || n < 0)
    return APIC_ERR_INVALID_ARG;
  if (mode != APIC_LOAD_VOLUME && mode != APIC_FLUX_SURFACE && mode != APIC_EXPLICIT) return APIC_ERR_INVALID_ARG;
  if (mode == APIC_EXPLICIT && !explicit_state && n > 0) return APIC_ERR_INVALID_ARG;
  if (n == 0) return APIC_OK;
  return S->precision == APIC_FP64 ? inject_impl<double>(S, instance, species, n, mode, explicit_state)
                                   : inject_impl<float>(S, instance, species, n, mode, explicit_state);
}

// ---------------------------------------------------------------------------
// Read-back.
// ---------------------------------------------------------------------------
extern "C" int apic_tallies(apic_sim* S, int32_t instance, apic_tallies_t* out) {
  if (!S || !out) return APIC_ERR_INVALID_ARG;
  if (instance < 0 || instance >= S->n_inst) return APIC_ERR_INVALID_ARG;
  if (S->status != APIC_OK) return S->status;  // sticky
  const Inst& I = S->inst[instance];
  // every copy into one pinned staging block, stream-ordered after the
  // steps, then a single synchronisation
  auto words = [](const Inst& J) {
    return (size_t)J.n_species * ((size_t)J.n2 * kTallyBinWords + kTallyStepWords);
  };
  const size_t o_stp = 0, o_sol = o_stp + sizeof(StepState), o_ps = o_sol + sizeof(SolverState);
  const size_t o_hist = o_ps + 2 * sizeof(PopState);
  if (!S->h_tally) {
    size_t most = 0;
    for (const Inst& J : S->inst) most = std::max(most, (size_t)J.hist_cap * kNH * sizeof(double) + words(J) * 8);
    S->h_tally_bytes = o_hist + most;
    if (!S->ck(cudaMallocHost(&S->h_tally, S->h_tally_bytes), "cudaMallocHost")) return S->status;
  }
  const size_t tw = words(I);
  const size_t nh = (size_t)I.hist_cap * kNH;
  double* hist = (double*)(S->h_tally + o_hist);
  unsigned long long* tfix = (unsigned long long*)(S->h_tally + o_hist + nh * sizeof(double));
  PopState* psd = (PopState*)(S->h_tally + o_ps);
  if (out->bins) S->d2h(tfix, S->d.tfix + I.bin_off, tw);
  S->d2h((StepState*)(S->h_tally + o_stp), S->d.stp + instance, 1);
  S->d2h((SolverState*)(S->h_tally + o_sol), S->d.sol + instance, 1);
  S->d2h(psd, S->d.ps + I.pop0, (size_t)I.n_species);  // the instance's populations are consecutive
  S->d2h(hist, S->d.hist + I.hist_off, nh);
  if (!S->sync()) return S->status;
  StepState stp;
  SolverState sol;
  std::memcpy(&stp, S->h_tally + o_stp, sizeof(stp));
  std::memcpy(&sol, S->h_tally + o_sol, sizeof(sol));
  PopState ps[2];
  std::memset(ps, 0, sizeof(ps));
  for (int s = 0; s < I.n_species; ++s) ps[s] = psd[s];
  if (out->bins) {
    // bins from the fixed-point sums (tally_fixed.cuh): charge = hits q w,
    // momenta and L_z times m w v_th, energy times m w v_th^2, plus the
    // binding energy per hit of a positive species
    for (int s = 0; s < I.n_species; ++s) {
      const Pop& P = S->pop[I.pop0 + s];
      const double mwu = P.m * P.w * P.tunit;
      for (int j = 0; j < I.n2; ++j) {
        const unsigned long long* b = tfix + (P.tfix_off - I.bin_off) + (size_t)j * kTallyBinWords;
        double* o = out->bins + ((size_t)s * I.n2 + j) * kNT;
        const double hits = (double)b[0];
        o[0] = hits;
        o[1] = hits * P.q * P.w;
        o[2] = mwu * fixed128_value(b[1], b[2]);
        o[3] = mwu * fixed128_value(b[3], b[4]);
        o[4] = mwu * fixed128_value(b[5], b[6]);
        o[5] = mwu * P.tunit * fixed128_value(b[7], b[8]);
        o[6] = o[5] + (P.q > 0.0 ? hits * I.e_bind * P.w : 0.0);
      }
    }
  }
  for (int s = 0; s < 2; ++s) {
    out->counts[s][0] = ps[s].loaded;
    out->counts[s][1] = ps[s].injected;
    out->counts[s][2] = ps[s].absorbed;
    out->counts[s][3] = ps[s].escaped;
    out->counts[s][4] = ps[s].loaded + ps[s].injected - ps[s].absorbed - ps[s].escaped - ps[s].dropped;
    out->counts[s][5] = ps[s].dropped;
  }
  out->step = stp.step;
  out->grain_Q = stp.Q;
  out->grain_FZ = stp.FZ;
  out->poisson_res = sol.res;
  out->poisson_iters = sol.iters;
  long long rows = std::min<long long>(stp.step, I.hist_cap);
  if (out->history) {
    long long cap = out->history_rows;
    long long w = std::min(rows, cap);
    long long first = stp.step - w;  // oldest row written
    for (long long r = 0; r < w; ++r) {
      long long src = (first + r) % I.hist_cap;
      std::memcpy(out->history + r * kNH, hist + src * kNH, sizeof(double) * kNH);
    }
    out->history_rows = w;
  } else {
    out->history_rows = rows;
  }
  return APIC_OK;
}

// ---- Checkpoint / resume --------------------------------------------------
// The state the next steps depend on: every population's live slots [0, n)
// of the five state arrays (the current particle buffer) and its free-slot
// stack, the population, solver and step scalars (counts, Philox draws
// consumed, injection carries, step index, grain charge), the node arrays
// carried from step to step (phi as the next solve's start, phi_prev, rho,
// the deposit accumulators of the last push and injection, the gradients and
// their pair table, the surface field), the fixed-point tallies and the
// history ring, and the host's step counter and sort interval.  Draws are
// counter-based (Philox on the population's draw count), so a resumed run
// draws what the uninterrupted one draws.
namespace {
constexpr unsigned long long kCkptMagic = 0x31504b4343495041ull;  // "APICCKP1"
struct CkptHeader {
  unsigned long long magic;
  int32_t version, precision, n_inst, n_pop;
  int64_t total_nodes, bins, hist, en, bytes;
  int64_t host_step, sorts, loop_iters;
  int32_t sort_interval, dirty;
};

struct CkptSizes {
  int64_t bins = 0, hist = 0, en = 0;
};

CkptSizes ckpt_sizes(const apic_sim* S) {
  CkptSizes z;
  for (const Inst& I : S->inst) {
    z.bins += (int64_t)I.n_species * ((int64_t)I.n2 * kTallyBinWords + kTallyStepWords);
    z.hist += (int64_t)I.hist_cap * kNH;
    z.en += I.N2;
  }
  return z;
}

// Bytes of a checkpoint whose populations hold ps[p].n slots and ps[p].n_holes free slots.
int64_t ckpt_bytes(const apic_sim* S, const PopState* ps) {
  const CkptSizes z = ckpt_sizes(S);
  const int64_t R = S->precision == APIC_FP64 ? 8 : 4, nodes = S->d.total_nodes;
  int64_t b = sizeof(CkptHeader) + (int64_t)sizeof(PopState) * S->n_pop +
              (int64_t)(sizeof(SolverState) + sizeof(StepState)) * S->n_inst;
  for (int p = 0; p < S->n_pop; ++p) b += ps[p].n * 5 * R + ps[p].n_holes * 4;
  b += 3 * 8 * nodes + 2 * 8 * nodes + 2 * R * nodes + (S->d.H ? 16 * nodes : 0);
  b += 8 * (z.bins + z.hist + z.en);
  return b;
}

// The node-sized and table arrays in checkpoint order: device pointer, bytes.
std::vector<std::pair<void*, int64_t>> ckpt_arrays(const apic_sim* S) {
  const CkptSizes z = ckpt_sizes(S);
  const DevPtrs& d = S->d;
  const int64_t R = S->precision == APIC_FP64 ? 8 : 4, nodes = d.total_nodes;
  std::vector<std::pair<void*, int64_t>> a = {
      {d.rho, 8 * nodes}, {d.phi, 8 * nodes}, {d.phi_prev, 8 * nodes}, {d.acc, 16 * nodes}, {d.G, 2 * R * nodes}};
  if (d.H) a.push_back({d.H, 16 * nodes});
  a.push_back({d.tfix, 8 * z.bins});
  a.push_back({d.hist, 8 * z.hist});
  a.push_back({d.en, 8 * z.en});
  return a;
}
}  // namespace

extern "C" int apic_checkpoint_size(apic_sim* S, int64_t* bytes) {
  if (!S || !bytes) return APIC_ERR_INVALID_ARG;
  if (S->status != APIC_OK) return S->status;
  std::vector<PopState> ps(S->n_pop);
  if (!S->d2h(ps.data(), S->d.ps, ps.size()) || !S->sync()) return S->status;
  *bytes = ckpt_bytes(S, ps.data());
  return APIC_OK;
}

extern "C" int apic_checkpoint_save(apic_sim* S, void* buf, int64_t bytes) {
  if (!S || !buf) return APIC_ERR_INVALID_ARG;
  if (S->status != APIC_OK) return S->status;
  std::vector<PopState> ps(S->n_pop);
  if (!S->d2h(ps.data(), S->d.ps, ps.size()) || !S->sync()) return S->status;
  const int64_t need = ckpt_bytes(S, ps.data());
  if (bytes < need) return APIC_ERR_INVALID_ARG;
  const CkptSizes z = ckpt_sizes(S);
  long long loops = 0;
  if (!S->d2h(&loops, S->d.cnt, 1) || !S->sync()) return S->status;
  CkptHeader h;
  std::memset(&h, 0, sizeof(h));
  h.magic = kCkptMagic;
  h.version = 1;
  h.precision = S->precision;
  h.n_inst = S->n_inst;
  h.n_pop = S->n_pop;
  h.total_nodes = S->d.total_nodes;
  h.bins = z.bins;
  h.hist = z.hist;
  h.en = z.en;
  h.bytes = need;
  h.host_step = S->host_step;
  h.sorts = S->sorts;
  h.loop_iters = loops;
  h.sort_interval = S->sort_interval;
  h.dirty = S->dirty ? 1 : 0;
  unsigned char* o = (unsigned char*)buf;
  std::memcpy(o, &h, sizeof(h));
  o += sizeof(h);
  std::memcpy(o, ps.data(), sizeof(PopState) * ps.size());
  o += sizeof(PopState) * ps.size();
  auto get = [&](const void* src, int64_t n) {
    if (n > 0) S->ck(cudaMemcpyAsync(o, src, (size_t)n, cudaMemcpyDeviceToHost, S->stream), "checkpoint D2H");
    o += n;
  };
  get(S->d.sol, (int64_t)sizeof(SolverState) * S->n_inst);
  get(S->d.stp, (int64_t)sizeof(StepState) * S->n_inst);
  const DevPtrs v = S->view(S->par);
  const int64_t R = S->precision == APIC_FP64 ? 8 : 4;
  void* arr[5] = {v.x1, v.x2, v.vR, v.vZ, v.vT};
  for (int p = 0; p < S->n_pop; ++p) {
    const Pop& P = S->pop[p];
    for (void* a : arr) get((const unsigned char*)a + P.base * R, ps[p].n * R);
    get(S->d.holes + P.base, ps[p].n_holes * 4);
  }
  for (const auto& a : ckpt_arrays(S)) get(a.first, a.second);
  if (!S->sync()) return S->status;
  return (int64_t)(o - (unsigned char*)buf) == need ? APIC_OK : S->fail(APIC_ERR_INVALID_ARG, "checkpoint layout");
}

extern "C" int apic_checkpoint_load(apic_sim* S, const void* buf, int64_t bytes) {
  if (!S || !buf || bytes < (int64_t)sizeof(CkptHeader)) return APIC_ERR_INVALID_ARG;
  if (S->status != APIC_OK) return S->status;
  CkptHeader h;
  std::memcpy(&h, buf, sizeof(h));
  const CkptSizes z = ckpt_sizes(S);
  if (h.magic != kCkptMagic || h.version != 1 || h.precision != S->precision || h.n_inst != S->n_inst ||
      h.n_pop != S->n_pop || h.total_nodes != S->d.total_nodes || h.bins != z.bins || h.hist != z.hist ||
      h.en != z.en || h.bytes > bytes || (h.sort_interval > 0) != (S->sort_interval > 0))
    return APIC_ERR_INVALID_ARG;
  const unsigned char* o = (const unsigned char*)buf + sizeof(h);
  std::vector<PopState> ps(S->n_pop);
  if ((int64_t)(sizeof(h) + sizeof(PopState) * ps.size()) > bytes) return APIC_ERR_INVALID_ARG;
  std::memcpy(ps.data(), o, sizeof(PopState) * ps.size());
  o += sizeof(PopState) * ps.size();
  for (int p = 0; p < S->n_pop; ++p)
    if (ps[p].n < 0 || ps[p].n > S->pop[p].cap || ps[p].n_holes < 0 || ps[p].n_holes > ps[p].n)
      return APIC_ERR_INVALID_ARG;
  if (ckpt_bytes(S, ps.data()) != h.bytes) return APIC_ERR_INVALID_ARG;
  if (!S->sync()) return S->status;  // nothing of this simulation in flight
  auto put = [&](void* dst, int64_t n) {
    if (n > 0) S->ck(cudaMemcpyAsync(dst, o, (size_t)n, cudaMemcpyHostToDevice, S->stream), "checkpoint H2D");
    o += n;
  };
  S->h2d(S->d.ps, ps.data(), ps.size());  // (the populations' scalars, read above)
  put(S->d.sol, (int64_t)sizeof(SolverState) * S->n_inst);
  put(S->d.stp, (int64_t)sizeof(StepState) * S->n_inst);
  const DevPtrs v = S->view(S->par);
  const int64_t R = S->precision == APIC_FP64 ? 8 : 4;
  void* arr[5] = {v.x1, v.x2, v.vR, v.vZ, v.vT};
  for (int p = 0; p < S->n_pop; ++p) {
    const Pop& P = S->pop[p];
    for (void* a : arr) put((unsigned char*)a + P.base * R, ps[p].n * R);
    put(S->d.holes + P.base, ps[p].n_holes * 4);
  }
  for (const auto& a : ckpt_arrays(S)) put(a.first, a.second);
  const long long loops = h.loop_iters;
  S->h2d(S->d.cnt, &loops, 1);
  if (!S->sync()) return S->status;  // (the host copies are pageable: complete before returning)
  S->host_step = h.host_step;
  S->sorts = h.sorts;
  if (h.sort_interval > 0) S->sort_interval = h.sort_interval;
  S->dirty = h.dirty != 0;
  return APIC_OK;
}

// Solve of instance inst for the right-hand side in d.b (with its |b|^2
// partials), from the guess in d.phi; the other instances keep their phi.
template <class Real>
static bool solve_instance(apic_sim* S, int inst) {
  DevPtrs& d = S->d;
  if (S->coop > 0) return S->ck(solve_coop<Real>(S, d, S->stream, 0, inst), "cooperative solve");
  launch_bicg_init<Real>(d, S->stream);
  int it = 0;
  SolverState sol;
  for (;;) {
    launch_bicg_iter<Real>(d, S->plan, S->stream);
    launch_bicg_check(d, 0, 0, S->stream);
    if (!S->d2h(&sol, d.sol + inst, 1) || !S->sync()) return false;
    if (sol.done || ++it > 1000) break;
  }
  return true;
}

template <class Real>
static int solve_impl(apic_sim* S, int inst, const double* rho, double* phi_out) {
  const Inst& I = S->inst[inst];
  DevPtrs& d = S->d;
  if (!S->ck(cudaMemcpyAsync(S->phi_save, d.phi, sizeof(double) * d.total_nodes, cudaMemcpyDeviceToDevice, S->stream),
             "save phi"))
    return S->status;
  if (rho && !S->h2d(d.rho + I.node_off, rho, (size_t)I.nodes)) return S->status;
  launch_b_from_rho(d, inst, S->stream);
  if (I.flags & APIC_BOLTZMANN) {  // Newton from the current phi
    for (int k = 0; k < S->newton; ++k) {
      launch_newton(d, inst, k == S->newton - 1 ? 0.0 : S->newton_eta, S->stream);
      if (!solve_instance<Real>(S, inst)) return S->status;
    }
    launch_newton_end(d, S->stream);
  } else if (!solve_instance<Real>(S, inst)) {
    return S->status;
  }
  if (phi_out) S->d2h(phi_out, d.phi + I.node_off, (size_t)I.nodes);
  S->ck(cudaMemcpyAsync(d.phi, S->phi_save, sizeof(double) * d.total_nodes, cudaMemcpyDeviceToDevice, S->stream),
        "restore phi");
  return read_status(S);
}

// Vacuum field of every isolated grain (APIC_FLOATING): the solve with no
// charge, phi = 1 on the grain and 0 on the outer surface, kept in phi_vac
// (its boundary rows included); each grain's potential starts at the
// configured one.  The step's phi is restored afterwards.
template <class Real>
static bool vacuum_fields(apic_sim* S) {
  DevPtrs& d = S->d;
  std::vector<StepState> st((size_t)S->n_inst);
  std::memset((void*)st.data(), 0, sizeof(StepState) * st.size());
  for (int k = 0; k < S->n_inst; ++k) st[k].phig = S->inst[k].phi_g;
  if (!S->h2d(d.stp, st.data(), st.size()) ||
      !S->ck(cudaMemcpyAsync(S->phi_save, d.phi, sizeof(double) * d.total_nodes, cudaMemcpyDeviceToDevice, S->stream),
             "save phi"))
    return false;
  for (int k = 0; k < S->n_inst; ++k) {
    const Inst& I = S->inst[k];
    if (!(I.flags & APIC_FLOATING)) continue;
    std::vector<double> hbg;
    grain_bbc(I, hbg);
    if (!S->h2d(d.bbc_g + I.node_off, hbg.data(), hbg.size())) return false;
    launch_b_vacuum(d, k, S->stream);
    if (!solve_instance<Real>(S, k)) return false;
    launch_store_vacuum(d, k, S->stream);
    if (!S->sync()) return false;  // hbg goes out of scope
  }
  return S->ck(cudaMemcpyAsync(d.phi, S->phi_save, sizeof(double) * d.total_nodes, cudaMemcpyDeviceToDevice, S->stream),
               "restore phi") &&
         S->ck(cudaGetLastError(), "vacuum field") && S->sync() && read_status(S) == APIC_OK;
}

extern "C" int apic_solve_poisson(apic_sim* S, int32_t instance, const double* rho, double* phi_out) {
  if (!S) return APIC_ERR_INVALID_ARG;
  if (S->status != APIC_OK) return S->status;
  if (instance < 0 || instance >= S->n_inst) return APIC_ERR_INVALID_ARG;
  if (S->inst[instance].flags & APIC_NO_FIELD) return APIC_ERR_INVALID_ARG;
  return S->precision == APIC_FP64 ? solve_impl<double>(S, instance, rho, phi_out)
                                   : solve_impl<float>(S, instance, rho, phi_out);
}

template <class Real>
static int particles_impl(apic_sim* S, int inst, int species, double* out, long long cap, long long* n_out) {
  int pop = S->inst[inst].pop0 + species;
  PopState ps;
  if (!S->sync() || !S->d2h(&ps, S->d.ps + pop, 1) || !S->sync()) return S->status;
  long long n = ps.n;
  std::vector<double> h((size_t)std::max<long long>(1, n) * 5);
  if (n > 0) {
    double* tmp = (double*)S->dalloc(sizeof(double) * 5 * (size_t)n);
    if (!tmp) return S->status;
    long long nn = n;
    launch_gather_particles<Real>(S->view(S->par), pop, tmp, &nn, S->stream);
    S->d2h(h.data(), tmp, 5 * (size_t)n);
    if (!S->sync()) return S->status;
    S->blocks.pop_back();
    if (S->have_alloc) S->alloc.free(tmp, (void*)S->stream, S->alloc.ctx);
    else cudaFreeAsync(tmp, S->stream);
  }
  long long w = 0;
  for (long long k = 0; k < n; ++k) {
    if (!(h[5 * k] < 0.0)) continue;  // freed slot
    if (w < cap && out) std::memcpy(out + 5 * w, h.data() + 5 * k, sizeof(double) * 5);
    ++w;
  }
  *n_out = std::min(w, cap);
  return APIC_OK;
}

extern "C" int apic_get_particles(apic_sim* S, int32_t instance, int32_t species, double* out, int64_t capacity,
                                  int64_t* n_out) {
  if (!S || !n_out) return APIC_ERR_INVALID_ARG;
  if (instance < 0 || instance >= S->n_inst || species < 0 || species >= S->inst[instance].n_species)
    return APIC_ERR_INVALID_ARG;
  long long n = 0;
  int rc = S->precision == APIC_FP64 ? particles_impl<double>(S, instance, species, out, capacity, &n)
                                     : particles_impl<float>(S, instance, species, out, capacity, &n);
  *n_out = n;
  return rc;
}

extern "C" int apic_get_field(apic_sim* S, int32_t instance, int32_t which, double* out) {
  if (!S || !out) return APIC_ERR_INVALID_ARG;
  if (instance < 0 || instance >= S->n_inst || which < 0 || which > 4) return APIC_ERR_INVALID_ARG;
  const Inst& I = S->inst[instance];
  if (!S->sync()) return S->status;
  if (which == 0) S->d2h(out, S->d.rho + I.node_off, (size_t)I.nodes);
  else if (which == 1) S->d2h(out, S->d.phi + I.node_off, (size_t)I.nodes);
  else if (which == 4) S->d2h(out, S->d.V + I.node_off, (size_t)I.nodes);
  else {
    size_t R = S->precision == APIC_FP64 ? 8 : 4;
    std::vector<unsigned char> g((size_t)I.nodes * 2 * R);
    S->ck(cudaMemcpyAsync(g.data(), (unsigned char*)S->d.G + (size_t)I.node_off * 2 * R, g.size(),
                          cudaMemcpyDeviceToHost, S->stream),
          "D2H");
    if (!S->sync()) return S->status;
    int c = which - 2;
    for (long long k = 0; k < I.nodes; ++k) {
      if (R == 8) out[k] = ((const double*)g.data())[2 * k + c];
      else out[k] = (double)((const float*)g.data())[2 * k + c];
    }
  }
  return S->sync() ? APIC_OK : S->status;
}

extern "C" const char* apic_last_error(const apic_sim* S) { return S ? S->msg.c_str() : "null simulation"; }

extern "C" int32_t apic_num_instances(const apic_sim* S) { return S ? S->n_inst : 0; }

// ---------------------------------------------------------------------------
// Sensitivity window: forward-mode derivatives of window-averaged outputs
// with respect to (alpha, phi_g, B).
// ---------------------------------------------------------------------------
using D1h = ad::Dual<double, 1>;

// Derivative tables of the set-up (node volumes, sampling tables, domain
// volume, the unscaled Eq. 7 rows) along alpha, from the same host code run
// on dual numbers; the phi_g Dirichlet term of the scaled system.
template <class Real>
static bool tangent_setup(apic_sim* S) {
  if (S->tan_ready) return true;
  if (!S->sync()) return false;
  TanPtrs& t = S->tan;
  const DevPtrs& d = S->d;
  const long long tn = d.total_nodes;
  const int ni = S->n_inst;
  const size_t R = sizeof(Real);
  t.stride = S->slots;
  t.ds = S->dalloc(R * 5 * kNPar * (size_t)S->slots);
  t.drho = (double*)S->dalloc(sizeof(double) * kNPar * tn);
  t.dphi = (double*)S->dalloc(sizeof(double) * kNPar * tn);
  t.bt = (double*)S->dalloc(sizeof(double) * kNPar * tn);
  t.phi0 = S->phi_save;
  t.dG = S->dalloc(2 * R * kNPar * tn);
  t.dV = (double*)S->dalloc(sizeof(double) * tn);
  t.dst = (double*)S->dalloc(sizeof(double) * kSt * tn);
  t.bbc_g = (double*)S->dalloc(sizeof(double) * tn);
  t.dtab = (double*)S->dalloc(sizeof(double) * S->tab_total);
  t.dlnw = (double*)S->dalloc(sizeof(double) * ni);
  t.tally = (double*)S->dalloc(sizeof(double) * ni * kNOut * kNPar);
  t.jac = (double*)S->dalloc(sizeof(double) * ni * kNOut * kNPar);
  t.vals = (double*)S->dalloc(sizeof(double) * ni * kNOut);
  if (S->status != APIC_OK) return false;
  std::vector<double> dlnw(ni);
  for (int k = 0; k < ni; ++k) {
    const Inst& I = S->inst[k];
    const D1h al = D1h::seed(I.alpha, 0);
    std::vector<D1h> tab;
    D1h vd, ao, ag;
    tables_t<D1h>(I, al, tab, vd, ao, ag);
    std::vector<double> htab(tab.size());
    for (size_t q = 0; q < tab.size(); ++q) htab[q] = tab[q].d[0];
    dlnw[k] = vd.d[0] / vd.v;
    std::vector<D1h> V;
    volumes_t<D1h>(I, al, V);
    std::vector<double> hV(V.size());
    for (size_t q = 0; q < V.size(); ++q) hV[q] = V[q].d[0];
    std::vector<double> hst((size_t)kSt * I.nodes, 0.0), hbg;
    for (int i = 1; i < I.n1; ++i)
      for (int j = 0; j <= I.n2; ++j) {
        size_t nd = (size_t)i * I.N2 + j;
        D1h wd[kSt];
        fine_row<D1h>(I, al, i, j, wd, V.data());
        for (int q = 0; q < kSt; ++q) hst[(size_t)q * I.nodes + nd] = wd[q].d[0];
      }
    grain_bbc(I, hbg);
    S->h2d(t.dtab + I.tab_off, htab.data(), htab.size());
    S->h2d(t.dV + I.node_off, hV.data(), hV.size());
    S->h2d(t.dst + (long long)kSt * I.node_off, hst.data(), hst.size());
    S->h2d(t.bbc_g + I.node_off, hbg.data(), hbg.size());
    if (!S->sync()) return false;  // host vectors go out of scope
  }
  S->h2d(t.dlnw, dlnw.data(), dlnw.size());
  if (!S->sync()) return false;
  S->tan_ready = true;
  return true;
}

// One Poisson solve of whatever right-hand side d.b holds, from the guess in d.phi.
template <class Real>
static bool solve_now(apic_sim* S, const DevPtrs& d) {
  if (S->coop > 0) return S->ck(solve_coop<Real>(S, d, S->stream), "cooperative solve");
  launch_bicg_init<Real>(d, S->stream);
  enqueue_solver_iterations_fixed<Real>(S, d, S->stream);
  return true;
}

template <class Real>
static int sensitivity_impl(apic_sim* S, int n, double* values, double* jac) {
  if (S->chord) return S->fail(APIC_ERR_INVALID_ARG, "the sensitivity window does not take APIC_CHORD_ABSORB");
  if (S->floating) return S->fail(APIC_ERR_INVALID_ARG, "the sensitivity window does not take APIC_FLOATING");
  if (S->boltz) return S->fail(APIC_ERR_INVALID_ARG, "the sensitivity window does not take APIC_BOLTZMANN");
  if (!tangent_setup<Real>(S)) return S->status;
  const TanPtrs& t = S->tan;
  const DevPtrs d = S->view(S->par);
  const long long tn = d.total_nodes;
  const int ni = S->n_inst;
  cudaStream_t s = S->stream;
  const size_t R = sizeof(Real);
  // the window starts from the current state, whose derivatives are zero
  S->ck(cudaMemsetAsync(t.ds, 0, R * 5 * kNPar * (size_t)S->slots, s), "memset");
  S->ck(cudaMemsetAsync(t.dphi, 0, sizeof(double) * kNPar * tn, s), "memset");
  S->ck(cudaMemsetAsync(t.tally, 0, sizeof(double) * ni * kNOut * kNPar, s), "memset");
  S->ck(cudaMemsetAsync(t.jac, 0, sizeof(double) * ni * kNOut * kNPar, s), "memset");
  S->ck(cudaMemsetAsync(t.vals, 0, sizeof(double) * ni * kNOut, s), "memset");
  for (int k = 0; k < n && S->status == APIC_OK; ++k) {
    // deposit of every particle (values and derivatives), charge density
    S->ck(cudaMemsetAsync(d.acc, 0, sizeof(unsigned long long) * 2 * tn, s), "memset");
    launch_deposit_all<Real>(d, S->push_grid, S->max_n2, s);
    S->ck(cudaMemsetAsync(t.drho, 0, sizeof(double) * kNPar * tn, s), "memset");
    launch_tan_deposit<Real>(d, t, S->push_grid, S->max_n2, s);
    launch_rho<Real>(d, s);
    launch_tan_rho(d, t, s);
    // Poisson: the step's problem, then the three tangent problems
    if (!solve_now<Real>(S, d)) break;
    S->ck(cudaMemcpyAsync(t.phi0, d.phi, sizeof(double) * tn, cudaMemcpyDeviceToDevice, s), "copy phi");
    if (S->plan.bcr.n_inst > 0 && kNPar <= kBcrMaxRhs && kNPar * ni <= kCoopMaxInst) {
      // the three tangent systems share the reduction's blocks: one launch
      BcrRhs rh{};
      rh.n = kNPar;
      for (int p = 0; p < kNPar; ++p) {
        launch_tan_b(d, t, p, 1, s);
        rh.slot[p] = kTanSlot + p;
        rh.x[p] = t.dphi + (long long)p * tn;
        rh.b[p] = t.bt + (long long)p * tn;
      }
      if (!S->ck(launch_solve_bcr_rhs(d, S->plan, S->coop, rh, s), "tangent solves")) break;
      for (int p = 0; p < kNPar; ++p) launch_tan_store(d, t, p, 1, s);
    } else {
      for (int p = 0; p < kNPar; ++p) {
        launch_tan_b(d, t, p, 0, s);
        if (!solve_now<Real>(S, d)) break;
        launch_tan_store(d, t, p, 0, s);
      }
    }
    S->ck(cudaMemcpyAsync(d.phi, t.phi0, sizeof(double) * tn, cudaMemcpyDeviceToDevice, s), "restore phi");
    // node gradients and surface quantities (the step's, then their derivatives)
    launch_gradients<Real>(d, s);
    launch_surface(d, s);
    for (int p = 0; p < kNPar; ++p) {
      DevPtrs dp = d;
      dp.phi = t.dphi + (long long)p * tn;
      dp.G = (char*)t.dG + (size_t)p * tn * 2 * R;
      launch_gradients<Real>(dp, s);
    }
    launch_tan_surface(d, t, s);
    // particles, injection, bookkeeping
    launch_tan_push<Real>(d, t, S->push_grid, s);
    launch_tan_inject<Real>(d, t, S->max_inj, s);
    launch_tan_step_end(d, t, s);
    launch_step_end(d, s);
    S->host_step += 1;
  }
  S->dirty = true;  // the accumulators no longer hold the current particles
  if (!S->ck(cudaGetLastError(), "sensitivity launch")) return S->status;
  std::vector<double> hv((size_t)ni * kNOut), hj((size_t)ni * kNOut * kNPar);
  S->d2h(hv.data(), t.vals, hv.size());
  S->d2h(hj.data(), t.jac, hj.size());
  int rc = read_status(S);
  if (rc != APIC_OK) return rc;
  for (size_t q = 0; q < hv.size(); ++q)
    if (values) values[q] = hv[q] / n;
  for (size_t q = 0; q < hj.size(); ++q)
    if (jac) jac[q] = hj[q] / n;
  return APIC_OK;
}

extern "C" int apic_sensitivity(apic_sim* S, int32_t n_steps, double* values, double* jacobian) {
  if (!S) return APIC_ERR_INVALID_ARG;
  if (S->status != APIC_OK) return S->status;
  if (n_steps < 1) return APIC_ERR_INVALID_ARG;
  return S->precision == APIC_FP64 ? sensitivity_impl<double>(S, n_steps, values, jacobian)
                                   : sensitivity_impl<float>(S, n_steps, values, jacobian);
}

// Reverse-sweep state for windows of up to K steps: checkpoints, fates,
// injection records, adjoint vectors, and a nested-dissection factorisation
// of every instance's solved operator in FP64 for the transposed solve.
template <class Real>
static bool adjoint_setup(apic_sim* S, int K) {
  if (!tangent_setup<Real>(S)) return false;
  AdjPtrs& a = S->adj;
  const DevPtrs& d = S->d;
  const long long tn = d.total_nodes;
  const int ni = S->n_inst;
  const size_t R = sizeof(Real);
  if (S->adj_K < K) {
    // (a smaller earlier allocation stays in the pool until apic_destroy)
    a.K = K;
    a.stride = S->slots;
    a.ck = S->dalloc(R * 5 * (size_t)K * (size_t)S->slots);
    a.ck_ps = (PopState*)S->dalloc(sizeof(PopState) * (size_t)(K + 1) * S->n_pop);
    a.ck_rho = (double*)S->dalloc(sizeof(double) * (size_t)K * tn);
    a.ck_phi = (double*)S->dalloc(sizeof(double) * (size_t)K * tn);
    a.fate = (uint8_t*)S->dalloc((size_t)K * (size_t)S->slots);
    a.inj_cap = std::max<long long>(1, S->max_inj);
    a.inj = (int64_t*)S->dalloc(sizeof(int64_t) * (size_t)K * S->n_pop * (size_t)a.inj_cap);
    if (!a.lam) {
      a.lam = (double*)S->dalloc(sizeof(double) * 5 * (size_t)S->slots);
      a.lG = (double*)S->dalloc(sizeof(double) * 2 * tn);
      a.lphi = (double*)S->dalloc(sizeof(double) * tn);
      a.lrho = (double*)S->dalloc(sizeof(double) * tn);
      a.Gk = S->dalloc(2 * R * tn);
      a.seed = (double*)S->dalloc(sizeof(double) * ni * kNOut);
      a.grad = (double*)S->dalloc(sizeof(double) * ni * kNPar);
      a.vals = (double*)S->dalloc(sizeof(double) * ni * kNOut);
    }
    if (S->status != APIC_OK) return false;
    S->adj_K = K;
  }
  if (a.nd_front) return true;
  // the transposed solve: every instance's operator (rows scaled as solved)
  // factored by nested dissection, FP64 fronts
  NdUpload up;
  std::vector<NdFactor> fs(ni);
  std::vector<int64_t> mat0(ni);
  int64_t mat = 0, w = 0, unk = 0;
  int T = (int)std::min<unsigned>(16u, std::max(1u, std::thread::hardware_concurrency()));
  S->adj_levels.assign(ni, {});
  S->adj_smem.assign(ni, 1);
  for (int k = 0; k < ni; ++k) {
    const Inst& I = S->inst[k];
    if (ni > kCoopMaxInst) {
      S->fail(APIC_ERR_INVALID_ARG, "too many instances for the reverse sweep");
      return false;
    }
    a.unk_off[k] = unk;
    unk += (long long)(I.n1 - 1) * I.N2;
    if (I.flags & APIC_NO_FIELD) continue;
    std::vector<double> V, rsc, bbc;
    build_volumes(I, V);
    HostLevel L;
    build_fine(I, V, L, rsc, bbc);
    std::string why;
    if (!nd_build(I.n1 - 1, I.N2, nd_coef, &L, 16, T, true, fs[k], why)) {
      S->fail(APIC_ERR_INVALID_ARG, "reverse sweep: " + why);
      return false;
    }
    const int f0 = (int)up.fronts.size();
    NdLevels lv;
    nd_layout(fs[k], mat, w, kNdWarpMaxS, kNdWarpMaxU, kNdWarpStage, kNdTaskFloats, kNdTaskRows, kNdTaskFronts,
              kNdUnitStage, 1, up, lv);
    mat0[k] = mat;
    mat += fs[k].fm_total + fs[k].nb_total;
    w += fs[k].w_total;
    auto& lvs = S->adj_levels[k];
    lvs.assign(fs[k].depth + 1, {0, 0});
    for (int q = f0; q < (int)up.fronts.size(); ++q) {
      const NdFront& F = up.fronts[q];
      auto& r = lvs[F.level];
      if (r.second == 0) r.first = q;
      r.second = q + 1;
      S->adj_smem[k] = std::max(S->adj_smem[k], F.s + F.u);
    }
  }
  a.unk_off[ni] = unk;
  a.rhs = (double*)S->dalloc(sizeof(double) * (size_t)std::max<int64_t>(1, unk));
  a.ndw = (double*)S->dalloc(sizeof(double) * (size_t)std::max<int64_t>(1, w));
  double* mbuf = (double*)S->dalloc(sizeof(double) * (size_t)std::max<int64_t>(1, mat));
  a.nd_front = (const NdFront*)S->dalloc(sizeof(NdFront) * std::max<size_t>(1, up.fronts.size()));
  a.nd_idx = (const int32_t*)S->dalloc(sizeof(int32_t) * std::max<size_t>(1, up.idx.size()));
  a.nd_gather = (const int32_t*)S->dalloc(sizeof(int32_t) * std::max<size_t>(1, up.gather.size()));
  if (S->status != APIC_OK) return false;
  a.nd_mat = mbuf;
  S->h2d((NdFront*)a.nd_front, up.fronts.data(), up.fronts.size());
  S->h2d((int32_t*)a.nd_idx, up.idx.data(), up.idx.size());
  S->h2d((int32_t*)a.nd_gather, up.gather.data(), up.gather.size());
  for (int k = 0; k < ni; ++k) {
    if (fs[k].fm64.empty()) continue;
    S->h2d(mbuf + mat0[k], fs[k].fm64.data(), fs[k].fm64.size());
    S->h2d(mbuf + mat0[k] + fs[k].fm_total, fs[k].nb64.data(), fs[k].nb64.size());
  }
  for (int k = 0; k < ni; ++k) {
    int need = S->adj_smem[k] * (int)sizeof(double);
    if (need > 48 * 1024 &&
        !S->ck(cudaFuncSetAttribute(adj_ndT_kernel(), cudaFuncAttributeMaxDynamicSharedMemorySize, need), "smem"))
      return false;
  }
  return S->sync();
}

// The reverse sweep of an n-step window: forward pass with checkpoints,
// then the steps backwards (adjoint.cu).
template <class Real>
static int adjoint_impl(apic_sim* S, int n, const double* dL_dout, double* values, double* grad) {
  if (S->chord) return S->fail(APIC_ERR_INVALID_ARG, "the adjoint window does not take APIC_CHORD_ABSORB");
  if (S->floating) return S->fail(APIC_ERR_INVALID_ARG, "the adjoint window does not take APIC_FLOATING");
  if (S->boltz) return S->fail(APIC_ERR_INVALID_ARG, "the adjoint window does not take APIC_BOLTZMANN");
  if (!adjoint_setup<Real>(S, n)) return S->status;
  const TanPtrs& t = S->tan;
  AdjPtrs a = S->adj;
  a.K = n;
  const DevPtrs d = S->view(S->par);
  const long long tn = d.total_nodes;
  const int ni = S->n_inst;
  cudaStream_t s = S->stream;
  const size_t R = sizeof(Real);
  const size_t pbytes = R * (size_t)S->slots;
  std::vector<double> seed((size_t)ni * kNOut);
  for (size_t q = 0; q < seed.size(); ++q) seed[q] = dL_dout[q] / n;
  S->h2d(a.seed, seed.data(), seed.size());
  S->ck(cudaMemsetAsync(a.grad, 0, sizeof(double) * ni * kNPar, s), "memset");
  S->ck(cudaMemsetAsync(a.vals, 0, sizeof(double) * ni * kNOut, s), "memset");
  S->ck(cudaMemsetAsync(a.inj, 0xff, sizeof(int64_t) * (size_t)n * S->n_pop * a.inj_cap, s), "memset");
  void* arr[5] = {d.x1, d.x2, d.vR, d.vZ, d.vT};
  // forward pass, checkpoint k holding the state at the start of step k
  for (int k = 0; k < n && S->status == APIC_OK; ++k) {
    for (int c = 0; c < 5; ++c)
      S->ck(cudaMemcpyAsync((char*)a.ck + ((size_t)k * 5 + c) * pbytes, arr[c], pbytes, cudaMemcpyDeviceToDevice, s),
            "checkpoint");
    S->ck(cudaMemcpyAsync(a.ck_ps + (size_t)k * S->n_pop, d.ps, sizeof(PopState) * S->n_pop, cudaMemcpyDeviceToDevice,
                          s),
          "checkpoint");
    S->ck(cudaMemsetAsync(d.acc, 0, sizeof(unsigned long long) * 2 * tn, s), "memset");
    launch_deposit_all<Real>(d, S->push_grid, S->max_n2, s);
    launch_rho<Real>(d, s);
    S->ck(cudaMemcpyAsync(a.ck_rho + (size_t)k * tn, d.rho, sizeof(double) * tn, cudaMemcpyDeviceToDevice, s), "ck");
    if (!solve_now<Real>(S, d)) break;
    S->ck(cudaMemcpyAsync(a.ck_phi + (size_t)k * tn, d.phi, sizeof(double) * tn, cudaMemcpyDeviceToDevice, s), "ck");
    launch_gradients<Real>(d, s);
    launch_surface(d, s);
    launch_adj_fwd_push<Real>(d, a, k, s);
    launch_adj_fwd_inject<Real>(d, a, t, k, S->max_inj, s);
    launch_adj_values(d, a, s);
    launch_step_end(d, s);
    S->host_step += 1;
  }
  S->ck(cudaMemcpyAsync(a.ck_ps + (size_t)n * S->n_pop, d.ps, sizeof(PopState) * S->n_pop, cudaMemcpyDeviceToDevice, s),
        "checkpoint");
  S->dirty = true;  // the accumulators no longer hold the current particles
  // reverse pass
  S->ck(cudaMemsetAsync(a.lam, 0, sizeof(double) * 5 * (size_t)S->slots, s), "memset");
  for (int k = n - 1; k >= 0 && S->status == APIC_OK; --k) {
    DevPtrs dg = d;  // the node gradients of step k from its potential
    dg.phi = a.ck_phi + (size_t)k * tn;
    dg.G = a.Gk;
    launch_gradients<Real>(dg, s);
    S->ck(cudaMemsetAsync(a.lG, 0, sizeof(double) * 2 * tn, s), "memset");
    S->ck(cudaMemsetAsync(a.lphi, 0, sizeof(double) * tn, s), "memset");
    launch_adj_rev_inject<Real>(d, a, t, k, S->max_inj, s);
    launch_adj_rev_push<Real>(d, a, t, k, s);
    launch_adj_surface(d, a, t, k, s);
    launch_adj_gradT(d, a, s);
    launch_adj_to_unknowns(d, a, s);
    for (int q = 0; q < ni; ++q) {
      const auto& lv = S->adj_levels[q];
      for (int l = (int)lv.size() - 1; l >= 0; --l)
        launch_adj_ndT(a, lv[l].first, lv[l].second, a.unk_off[q], S->adj_smem[q], true, s);
      for (int l = 0; l < (int)lv.size(); ++l)
        launch_adj_ndT(a, lv[l].first, lv[l].second, a.unk_off[q], S->adj_smem[q], false, s);
    }
    launch_adj_after_solve(d, a, t, k, s);
    launch_adj_rev_deposit<Real>(d, a, k, s);
  }
  if (!S->ck(cudaGetLastError(), "adjoint launch")) return S->status;
  std::vector<double> hv((size_t)ni * kNOut), hg((size_t)ni * kNPar);
  S->d2h(hv.data(), a.vals, hv.size());
  S->d2h(hg.data(), a.grad, hg.size());
  int rc = read_status(S);
  if (rc != APIC_OK) return rc;
  for (size_t q = 0; q < hv.size(); ++q)
    if (values) values[q] = hv[q] / n;
  for (size_t q = 0; q < hg.size(); ++q)
    if (grad) grad[q] = hg[q];
  return APIC_OK;
}

extern "C" int apic_adjoint_window(apic_sim* S, int32_t n_steps, const double* dL_dout, double* values,
                                   double* grad) {
  if (!S || !dL_dout || !grad) return APIC_ERR_INVALID_ARG;
  if (S->status != APIC_OK) return S->status;
  if (n_steps < 1) return APIC_ERR_INVALID_ARG;
  return S->precision == APIC_FP64 ? adjoint_impl<double>(S, n_steps, dL_dout, values, grad)
                                   : adjoint_impl<float>(S, n_steps, dL_dout, values, grad);
}

extern "C" int apic_adjoint(apic_sim* S, int32_t n_steps, const double* dL_dout, double* grad) {
  return apic_adjoint_window(S, n_steps, dL_dout, nullptr, grad);
}
