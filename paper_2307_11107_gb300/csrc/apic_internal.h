// Internal data layout of libapic (host and device).  Not part of the ABI.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/apic.h"
#include "nd_factor.h"
#include "tally_fixed.cuh"

namespace apic {

constexpr int kNT = APIC_NT;
constexpr int kNH = APIC_NH;
// Inexact Newton (Boltzmann electrons): every Newton iteration but the last
// solves its linear system only until the residual has fallen by this factor
// (or below the tolerance); quadratic convergence makes up for it.  The
// environment knob APIC_NEWTON_ETA replaces it at creation.
constexpr double kNewtonEta = 1e-3;
constexpr int kMaxLevels = 12;
constexpr int kMaxPop = 128;      // populations (instance x species) per batch
constexpr int kTable = 4096;      // intervals of the inverse-CDF sampling tables
constexpr int kRedBlocks = 64;    // CTAs per instance in node-parallel kernels (fixed => deterministic sums)
constexpr int kNRed = 8;          // reduction slots per CTA
constexpr int kMaxCoarse = 2200;  // coarsening stops at the first level with at most this many unknowns
constexpr int kMaxDense = 9000;   // largest coarsest level accepted (its dense inverse is kept on the GPU)

// error bits of the device status word
constexpr int kErrCapacity = 1;
constexpr int kErrNotConverged = 2;
constexpr int kErrNonFinite = 4;
constexpr int kErrTimeout = 8;
constexpr unsigned long long kWaitNs = 2000000000ull;  // grid-barrier waits give up after 2 s
constexpr int kCoopMaxBlocks = 256;  // CTAs of the cooperative solver (partial-sum slots)
constexpr int kCoopMaxInst = 64;     // instances the cooperative solver handles

// One multigrid level of one instance.  Unknowns are the nodes of rows
// i = 1..n1-1 (all j); rows 0 and n1 hold Dirichlet values.
struct Level {
  int n1, n2, N1, N2;    // cells and nodes
  int64_t off;           // offset of this level's node vectors in the level pool
  int64_t st;            // offset of its stencil (kSt arrays of `nodes` entries)
  int pole_extra;        // 1 on the finest level: pole rows reach j +- 2
  int pad;
  int64_t fac[2];        // offsets of the line factorisations (x1-lines, x2-lines) in the factor pool
};

// Stencil slots: (di, dj) in {-1,0,1}^2 as 3*(di+1) + (dj+1), then the two
// pole reaches (j=0 -> j=2, j=n2 -> j=n2-2).
constexpr int kSt = 11;
__host__ __device__ constexpr int st_slot(int di, int dj) { return 3 * (di + 1) + (dj + 1); }
constexpr int kStPole = 9;  // coefficient of phi(i, 2) in row (i, 0) and of phi(i, n2-2) in row (i, n2)

struct Inst {
  double alpha, x1_out, phi_g, phi_out, B, dt, e_bind;
  double h1, h2;
  double V_dom, A_out, A_grain;
  double tol;
  double i2h1, i2h2;       // 1 / (2 h1), 1 / (2 h2) (central differences without a division per node)
  uint64_t seed;
  int n1, n2, N1, N2;
  int64_t nodes;           // N1 * N2
  int64_t node_off;        // offset into per-node arrays of the batch
  int64_t tab_off;         // offset of the two CDF tables (volume, surface), (kTable+1) each
  int64_t bin_off;         // first word of its populations' fixed-point tallies (Pop::tfix_off)
  int64_t hist_off;        // offset of the history ring [hist_cap][kNH]
  int64_t en_off;          // offset of the surface field E_n [N2] (and of the surface geometry, 4 per node)
  int32_t hist_cap;
  int32_t n_species;
  int32_t pop0;            // first population of this instance
  int32_t tag;             // Philox counter tag (user instance id)
  int32_t flags;
  int32_t max_iter;
  int32_t n_levels;
  int32_t tail_level;      // first level handled by the single-CTA tail kernel
  int64_t cinv_off;        // dense inverse of the coarsest level [coarse_n]^2
  int32_t coarse_n;
  int32_t guess;           // 1: start each solve from 2 phi^n - phi^(n-1)
  Level lv[kMaxLevels];
};

struct Pop {
  double q, m, T, w, vth, lam;
  double dep_scale;        // q * w * 2^-fbits
  int64_t base, cap;       // particle slots [base, base + cap)
  int32_t inst, species;
  int32_t fbits;           // fixed-point fraction bits of the deposit
  int32_t pad;
  int64_t acc_off;         // offset of this population's deposit accumulator (nodes of its instance)
  int64_t cell_off;        // first sort bin of this population (bins = grid rows)
  int64_t cells;           // sort bins of this population (n1 rows)
  double tunit;            // velocity unit of the fixed-point tallies (v_th)
  int64_t tfix_off;        // first word of its fixed-point tallies: [n2][kTallyBinWords], then [kTallyStepWords]
};

// Device-mutable counters of one population.
struct PopState {
  long long n;             // slots in use [0, n)
  long long n_holes;       // free slots stacked in `holes`
  long long draws;         // Philox draws consumed
  long long loaded, injected, absorbed, escaped, dropped;
  long long n_inj;         // surface injections of the current step
  long long inj_stored;    // of which stored this step
  double carry;            // fractional injection carry
  long long pad[5];
};

// Per-instance solver scalars (device).
struct SolverState {
  double rho, alpha, omega, rho_old;
  double eta2, rn0;         // inexact Newton: stop also at |r|^2 <= eta2 |r_0|^2 (0: the tolerance alone); |r_0|^2
  double res;              // relative residual of the last iterate
  int32_t iters, done;
  double pad[8];
};

// Per-instance step scalars (device).
struct StepState {
  long long step;
  double Q, FZ;            // grain charge and electric force of the last solve
  double tally[5];         // this step: charge, p_Z, L_z, heat, events (from the fixed-point sums at the step's end)
  // isolated grain (APIC_FLOATING): potential of the last field, the grain
  // charge it holds, the last correction, whether qg has been fixed yet
  double phig, qg, dphig, qg_set;
  double pad[2];
};

struct BcrInst;

// Pointers handed to every kernel.
struct DevPtrs {
  const Inst* inst;
  const Pop* pop;
  PopState* ps;
  SolverState* sol;
  StepState* stp;
  int n_inst, n_pop;
  int32_t* err;
  long long* cnt;                 // [0] Krylov-loop iterations executed (all steps); [1] the push's next chunk group
  // particles (element type = the precision of the batch)
  void *x1, *x2, *vR, *vZ, *vT;
  void *y1, *y2, *yR, *yZ, *yT;  // second buffer (sort)
  int32_t* holes;
  unsigned* cell_cnt;             // sort: particles per global cell
  unsigned long long* cell_off;   // sort: exclusive prefix over cells (size cells + 1)
  unsigned long long* scan_tmp;   // sort: block sums of the scan
  int64_t total_cells;
  // per-node FP64 arrays
  double *rho, *phi, *phi_prev, *V, *bbc, *rscale;
  double* Vinv;                   // 1 / V (the density without a division per node)
  double* bbc_g;                  // Dirichlet term of phi = 1 on the grain, 0 outside (APIC_FLOATING; else null)
  double* phi_vac;                // vacuum field of that problem, boundary rows included (APIC_FLOATING)
  double* diag0;                  // diagonal of the linear FP64 operator st64 (APIC_BOLTZMANN; else null)
  double *b, *r, *rh, *p, *v, *s, *t, *ph, *sh;
  double* st64;                   // finest-level stencil, FP64 [kSt][nodes] per instance (same offsets)
  unsigned long long* acc;        // deposit accumulators
  void* G;                        // node gradients (dphi/dx1, dphi/dx2) as pairs of the particle type
  float* H;                       // FP32: (G[n], G[n + 1]) per node n, four floats (the vector push's
                                  // gather reads a cell's four corners in two loads); null in FP64
  // multigrid (particle type)
  void* st;                       // stencils of all levels
  void *e, *f;                    // level vectors
  void* cinv;                     // coarsest inverses
  void* fac;                      // line factorisations of every level
  // tables and diagnostics (FP64)
  double* tab;
  int32_t* guide;                 // per table entry g: interval of (g / kTable) * total (same layout as tab)
  double* sgeo;                   // grain-surface geometry per x2 node: |grad x1|, n_Z, dA/dx2, trapezoid weight
  unsigned long long* tfix;       // fixed-point tallies of every population (tally_fixed.cuh)
  double* hist;
  double* en;
  double* red;                    // reduction partials [n_inst][kNRed][kRedBlocks]
  double* cred;                   // cooperative solver partials [n_inst][kNRed][kCoopMaxBlocks]
  unsigned* bar;                  // grid barrier of the cooperative solver (count, generation)
  unsigned long long wait_ns;     // time limit of a grid-barrier wait (global timer), then APIC_ERR_TIMEOUT
  int64_t total_nodes;
  int64_t level_nodes;
  // block cyclic reduction: factor blocks and tail inverses of every instance,
  // reduced right-hand side and correction rows, per-instance tables, phase schedule
  float* bcr;
  float* bcr_f;
  float* bcr_e;
  const BcrInst* bcr_inst;        // [n_inst]
  const int32_t* bcr_kind;        // [phases][n_inst]: kind << 8 | level of instance k's tasks in a phase (0: none)
  const int32_t* bcr_pre;         // [phases][n_inst + 1]: prefix sums of the instances' task counts
  const int32_t* bcr_npre;        // [n_inst + 1]: prefix sums of the instances' partial-sum ranges (kBcrSub nodes)
  const int32_t* bcr_tpre;        // [n_inst + 1]: prefix sums of the instances' node tasks
  double* bcr_part;               // [1 + kBcrMaxRhs][chunks]: |b|^2, then |r|^2 per right-hand side, of each range
  // nested dissection (instances with BcrInst::nd): fronts of every such
  // instance (offsets global: idx, gather, matrices in bcr, update vectors
  // per right-hand side in nd_w), their index and gather tables, the tasks
  // (front or first front, first row or front count, rows, 1 = one front per warp)
  const NdFront* nd_front;
  const int32_t* nd_idx;
  const int32_t* nd_gather;
  const int4* nd_task;
  const longlong2* nd_trange;  // per task: its matrix floats [x, y) in bcr (one contiguous range)
  float* nd_w;
  // dataflow sweeps (BcrPlan::nd_flow): the forward then the backward task
  // order (task, instance; every task after the tasks it depends on), the
  // tasks each front takes per sweep [2][fronts] and the done counters
  // [2][kBcrMaxRhs][fronts]
  const int2* nd_flow;
  const int32_t* nd_need;
  unsigned* nd_done;
};

#ifdef __CUDACC__
// This step's tallies of instance `inst` from its populations' fixed-point
// sums, in population order: charge, p_Z, L_z, heat (E_kin + E_bind), events.
__device__ inline void step_tallies(const DevPtrs& d, int inst, double out[5]) {
  const Inst& I = d.inst[inst];
  for (int k = 0; k < 5; ++k) out[k] = 0.0;
  for (int s = 0; s < I.n_species; ++s) {
    const Pop& P = d.pop[I.pop0 + s];
    const unsigned long long* st = d.tfix + P.tfix_off + (long long)I.n2 * kTallyBinWords;
    const double hits = (double)st[0], mwu = P.m * P.w * P.tunit;
    out[0] += hits * P.q * P.w;
    out[1] += mwu * fixed128_value(st[1], st[2]);
    out[2] += mwu * fixed128_value(st[3], st[4]);
    out[3] += mwu * P.tunit * fixed128_value(st[5], st[6]) + (P.q > 0.0 ? hits * I.e_bind * P.w : 0.0);
    out[4] += hits;
  }
}
#endif

// ---- sensitivity window (forward mode) ----
// Derivatives with respect to kNPar parameters, index p: 0 = alpha, 1 = phi_g,
// 2 = B.  Outputs, index o: 0 = drag F_Z (absorbed Z momentum per time),
// 1 = electric F_Z on the grain, 2 = current, 3 = torque T_z, 4 = grain charge Q.
constexpr int kNPar = 3;
constexpr int kNOut = 5;

struct TanPtrs {
  void* ds;                // particle tangents: component 5 p + c (c: x1, x2, vR, vZ, vTheta) of slot s at [comp * stride + s]
  int64_t stride;          // particle slots of one component (all populations)
  double* drho;            // [kNPar][total_nodes]: sum of q w dW, then d rho
  double* dphi;            // [kNPar][total_nodes]
  double* phi0;            // primal phi (all nodes) while the tangent systems are solved
  double* bt;              // [kNPar][total_nodes]: right-hand sides of the tangent systems (solved together)
  void* dG;                // [kNPar][total_nodes] node-gradient pairs in the particle type
  double* dV;              // d V_node / d alpha
  double* dst;             // d (unscaled Eq. 7 row, all kSt slots, Dirichlet neighbours kept) / d alpha [kSt][total_nodes]
  double* bbc_g;           // Dirichlet term of phi_g = 1, phi_out = 0 (rows scaled as the solved system)
  double* dtab;            // d (sampling tables) / d alpha, same layout as DevPtrs::tab
  double* dlnw;            // per instance: d ln w / d alpha = (d V_dom / d alpha) / V_dom
  double* tally;           // per instance [kNOut][kNPar]: this step's derivative tallies
  double* jac;             // per instance [kNOut][kNPar]: sums over the window
  double* vals;            // per instance [kNOut]: sums of the outputs over the window
};

// ---- reverse sweep (adjoint window) ----
// The forward pass of a K-step window keeps, per step k, the particle state
// and population counters at the start of the step, the step's rho and phi,
// each slot's fate in the push and each injection draw's slot; the reverse
// pass then runs the step's operations backwards, from step K-1 to 0.
struct AdjPtrs {
  int K;                   // window steps
  int pad;
  int64_t stride;          // particle slots of one component (all populations)
  void* ck;                // [K][5][stride] particle state at the start of step k (particle precision)
  PopState* ck_ps;         // [K + 1][n_pop] population counters at the start of step k (k = K: after the window)
  double* ck_rho;          // [K][total_nodes]
  double* ck_phi;          // [K][total_nodes]
  uint8_t* fate;           // [K][stride]: 0 kept, 1 absorbed, 2 escaped, 3 no live particle at the start of the step
  int64_t* inj;            // [K][n_pop][inj_cap]: slot (from the population's base) of injection draw q of step k;
                           // -1 absorbed during its first flight, -2 escaped
  int64_t inj_cap;
  double* lam;             // [5][stride] adjoint of the particle state
  double* lG;              // [2][total_nodes] adjoint of the node gradients
  double* lphi;            // [total_nodes] adjoint of phi
  double* lrho;            // [total_nodes] adjoint of rho
  double* rhs;             // transposed solve: right-hand side / solution over every instance's unknowns
  double* ndw;             // its update vectors
  void* Gk;                // node gradients of step k (pairs of the particle type)
  double* seed;            // [n_inst][kNOut] dL / d(output of one step) = dL_dout / K
  double* grad;            // [n_inst][kNPar] parameter adjoints
  double* vals;            // [n_inst][kNOut] window sums of the outputs
  // transposed nested-dissection solve: FP64 fronts of every instance
  const NdFront* nd_front;
  const int32_t* nd_idx;
  const int32_t* nd_gather;
  const double* nd_mat;
  int64_t unk_off[kCoopMaxInst + 1];  // first unknown of each instance in rhs
};
constexpr int kAdjBlocks = 256;  // CTAs of the reverse particle kernels (fixed: deterministic partial sums)

// ---- launchers (defined in the kernel translation units) ----
template <class Real>
void launch_load(const DevPtrs& d, int pop, long long n0, long long count, long long draw0, int kind,
                 cudaStream_t s);
template <class Real>
void launch_explicit(const DevPtrs& d, int pop, long long n0, long long count, const double* dstate,
                     cudaStream_t s);
template <class Real>
void launch_deposit_all(const DevPtrs& d, int max_grid, int max_n2, cudaStream_t s);
#ifndef APIC_PUSH4_MIN_BLOCKS
#define APIC_PUSH4_MIN_BLOCKS 3  // CTAs of the vector push per SM (80 registers: the four particles stay in registers)
#endif
// win_rows, chunk_group, chunk_items: the deposit window's node rows, the
// chunks a CTA takes per group and the particles per thread of a chunk of the
// vector push (16 or 32; 0: the defaults, push_window_rows, 4 and 32 when
// `particles` (the batch's particle slots) give every CTA two dozen chunks)
template <class Real>
void launch_push(const DevPtrs& d, int grid, int max_n2, bool chord, int win_rows, int chunk_group, int chunk_items,
                 long long particles, cudaStream_t s);
// Node rows of the push's shared-memory deposit window for grids up to max_n2
// cells in x2 (queried once per width; call at set-up, before any capture).
template <class Real>
int push_window_rows(int max_n2);
template <class Real>
void launch_inject(const DevPtrs& d, long long max_inj, cudaStream_t s);
// The particle sort (count, scan, scatter) for grids of up to max_rows cell
// rows; sort_setup queries its passes' occupancy once per row count (call at
// set-up, before any capture).
template <class Real>
void sort_setup(int max_rows);
template <class Real>
void launch_sort(const DevPtrs& d, int grid, int max_rows, cudaStream_t s);
template <class Real>
void launch_gather_particles(const DevPtrs& d, int pop, double* out, long long* n_out, cudaStream_t s);

// fields (fields.cu)
template <class Real>
void launch_rho(const DevPtrs& d, cudaStream_t s);
template <class Real>
void launch_gradients(const DevPtrs& d, cudaStream_t s);
void launch_surface(const DevPtrs& d, cudaStream_t s);
void launch_step_end(const DevPtrs& d, cudaStream_t s);
void launch_b_from_rho(const DevPtrs& d, int inst, cudaStream_t s);
void launch_b_vacuum(const DevPtrs& d, int inst, cudaStream_t s);
void launch_store_vacuum(const DevPtrs& d, int inst, cudaStream_t s);
void launch_float_phi(const DevPtrs& d, cudaStream_t s);
void launch_newton(const DevPtrs& d, int only, double eta, cudaStream_t s);
void launch_newton_end(const DevPtrs& d, cudaStream_t s);

// Block cyclic reduction (bcr.cu) of the finest-level system of every
// instance of a batch.  Instance k has the unknown rows i = 1..M (M = n1 - 1)
// of N = N2 unknowns each; rows beyond M carry a zero correction and are
// neither stored nor visited, so n1 need not be a power of two (K is the
// smallest with 2^K >= n1).  Reduction level l = 1..Lt (row stride
// h = 2^(l-1)) eliminates the rows k = h (2q + 1) <= M and keeps
// i = 2h (q + 1) <= M.
//   Level 1 (unless dense1): the x1 couplings A_i, C_i of Eq. 7 are
//   tridiagonal in j, so only B_k^-1 is stored.  Forward: y_k = B_k^-1 f_k, then f_i -= A_i y_{i-1} +
//   C_i y_{i+1} with the stencil's A_i, C_i.  Back: e_k = B_k^-1 (f_k - A_k
//   e_{k-1} - C_k e_{k+1}).
//   Level >= 2, and level 1 with dense1 (dense blocks):
//     kept row i:       P = A_i B_{i-h}^-1,  Q = C_i B_{i+h}^-1   (forward: f_i -= P f_{i-h} + Q f_{i+h})
//     eliminated row k: B_k^-1, G = B_k^-1 A_k, H = B_k^-1 C_k    (back: e_k = B_k^-1 f_k - G e_{k-h} - H e_{k+h})
// Blocks are FP32, column-major N x N with column stride Np (16-byte aligned
// columns); a block whose neighbour row is beyond M is zero.  The
// tail_m = M >> Lt rows left after level Lt (i = 2^Lt (q + 1)) form a block
// tridiagonal system of tail_n = tail_m N unknowns whose dense inverse (FP32,
// row-major, row stride tail_np, set up in FP64) is applied in one phase, in
// chunks of tail_rows rows; Lt is the fewest levels that bring tail_n under
// kBcrTailMax.
constexpr int kBcrMaxK = 13;
constexpr int kBcrMaxN = 256;       // blocks up to this size use the narrow solve kernel
constexpr int kBcrMaxNWide = 544;   // the wide one (17 outputs per lane): grids up to 543 cells in x2
constexpr int kBcrTailMax = 2048;
constexpr double kBcrMaxBytes = 24.0 * 1024 * 1024 * 1024;  // FP32 blocks of a whole batch held on the device
constexpr int kBcrUpdRows = 4;       // level-1 kept rows per update task
constexpr int kBcrSub = 256;         // nodes per partial sum of the node phases (density, residual)
constexpr int kBcrMaxTaskSub = 8;    // partial-sum ranges per node task at most
// task kinds of a phase of one instance
constexpr int kBcrFwd1 = 1;   // y_k = B_k^-1 f_k, level-1 eliminated rows
constexpr int kBcrUpd1 = 2;   // f_i -= A_i y_{i-1} + C_i y_{i+1}, level-1 kept rows
constexpr int kBcrFwd = 3;    // f_i -= P f_{i-h} + Q f_{i+h}, level >= 2
constexpr int kBcrTail = 4;   // e = T^-1 f on a chunk of tail rows
constexpr int kBcrBack = 5;   // e_k = B_k^-1 f_k - G e_{k-h} - H e_{k+h}, level >= 2
constexpr int kBcrBack1 = 6;  // e_k = B_k^-1 (f_k - A_k e_{k-1} - C_k e_{k+1}), level 1
// Nested dissection (nd_factor.h) in place of the reduction, per instance:
// the forward sweep from the deepest tree level to the root, then the
// backward sweep from the root down, one level per phase.
constexpr int kNdFwd = 7;     // a front's z_S = F_SS^-1 v_S and W = v_U - (F_US F_SS^-1) v_S
constexpr int kNdBack = 8;    // x_S = z_S - (F_SS^-1 F_SU) x_U, and x += e
constexpr int kNdMaxDepth = 40;
constexpr int kNdWarpMaxS = 64;     // fronts with a separator up to this size run one per warp
constexpr int kNdWarpMaxU = 192;    // ... and an update set up to this size
#ifndef APIC_ND_UNITS
#define APIC_ND_UNITS 4
#endif
// The dataflow sweeps split each solve CTA (16 warps) into kNdUnits workers,
// each with its own task; the task limits follow from a worker's share.
constexpr int kNdUnits = APIC_ND_UNITS;
constexpr int kNdWarpStage = 2048;    // matrix floats of a warp's front (staged in shared memory) at most
constexpr int kNdStageFloats = 16 * kNdWarpStage;  // the CTA's stage
constexpr int kNdUnitStage = kNdStageFloats / kNdUnits;  // a task's staged matrix rows at most
constexpr int kNdTaskFloats = kNdUnitStage;  // matrix floats per task of a large front (row chunks)
constexpr int kNdTaskFronts = 16 / kNdUnits;  // small fronts per task at most (one per warp of a worker)
constexpr int kNdTaskRows = 2048 / kNdUnits;  // rows per task of a large front at most
static_assert((kNdUnits == 1 || kNdUnits == 2 || kNdUnits == 4 || kNdUnits == 8) &&
                  kNdWarpStage * kNdTaskFronts <= kNdUnitStage,
              "workers of whole warps; tasks stage whole in a worker's stage");
struct BcrInst {
  int K;                    // 2^K >= n1
  int N;                    // block size N2
  int Np;                   // column stride (N rounded up to 4 floats)
  int Lt;                   // reduction levels before the dense tail (0..K-1)
  int M;                    // unknown rows (n1 - 1)
  int tail_m;               // rows of the tail system
  int tail_n;               // its unknowns (tail_m * N)
  int tail_np;              // row stride of the tail inverse (tail_n rounded up to 4 floats)
  int tail_rows;            // tail-inverse rows per task
  int smem;                 // 1: a task's blocks are staged in shared memory by bulk async copies
  int dense1;               // 1: level 1 stores P, Q, G, H too (one phase fewer per pass, more bytes)
  int64_t blk;              // floats per block (N * Np)
  int64_t base;             // first float of this instance's blocks in DevPtrs::bcr
  int64_t tail;             // first float of its tail inverse in DevPtrs::bcr
  int64_t foff;             // first float of its rows in bcr_f / bcr_e (M * N floats each)
  int64_t node_off;         // the instance's node offset (Inst::node_off)
  int64_t nodes;            // its nodes (Inst::nodes)
  int64_t st_off;           // offset of its finest-level FP32 stencil (Inst::lv[0].st)
  int64_t P[kBcrMaxK], Q[kBcrMaxK];                  // block index (from base) of the first block of each kind at level l
  int64_t Binv[kBcrMaxK], G[kBcrMaxK], H[kBcrMaxK];
  int64_t blocks;           // blocks of this instance
  int nd;                   // 1: nested dissection instead of the reduction (the fields above unused)
  int nd_depth;             // deepest tree level
  int32_t nd_ft[kNdMaxDepth + 2];  // forward tasks of level l: DevPtrs::nd_task [nd_ft[l], nd_ft[l + 1])
  int32_t nd_bt[kNdMaxDepth + 2];  // backward tasks of level l: [nd_bt[l], nd_bt[l + 1])
};
// Phase schedule: instance k runs its stages Fwd1, Upd1, Fwd(2..Lt), Tail,
// Back(Lt..2), Back1 (Lt = 0: Tail alone) in phases 0, 1, ..., one grid
// barrier after each phase.
struct BcrPlan {
  int n_inst;               // 0: not in use
  int phases;               // phases of one reduction pass
  int smem;                 // 1: dynamic shared memory holds staged blocks
  int resident;             // 1: the whole reduction fits in L2 (dense level 1, blocks staged in shared memory)
  int dyn;                  // dynamic shared memory bytes of the solve kernel
  int wide;                 // solve kernel: 0 narrow reduction, 1 wide reduction (some block larger than
                            // kBcrMaxN, or reduction and nested dissection), 2 nested dissection alone
  int64_t bytes;            // device bytes of all blocks and tail inverses
  int64_t chunks;           // partial-sum ranges of all instances (kBcrSub nodes each)
  int64_t rows;             // floats of one right-hand side's rows in bcr_f / bcr_e (all instances)
  int task_sub;             // partial-sum ranges per node task (1..kBcrMaxTaskSub)
  int pad2;
  int64_t nd_wrows;         // floats of one right-hand side's update vectors in nd_w (all instances)
  int nd_floats;            // shared-memory floats a large nested-dissection front needs (0: none)
  int nd_flow;              // 1: every instance by nested dissection, each sweep one dataflow phase
  int nd_nf, nd_nb;         // entries of the forward and backward task orders
  int nd_fronts;            // fronts of all instances
  int pad3;
};

// Poisson (poisson.cu): host-side launch plan of the multigrid levels.
struct SolvePlan {
  int max_tail;                   // levels run by the multi-CTA kernels (0 .. max_tail-1)
  int x1_blocks[kMaxLevels];      // grid.x of the x1-line kernels (lines per colour / warps per CTA)
  int x2_blocks[kMaxLevels];
  int x1_k[kMaxLevels];           // rows per lane of the warp line solver
  int x2_k[kMaxLevels];
  int node_blocks[kMaxLevels];    // grid.x of node-parallel kernels on each level
  int tail_threads, tail_k;
  int tail_bytes;                 // dynamic shared memory of the tail kernel
  int smooth_split;               // 1: pre-smoothing x1-lines only, post-smoothing x2-lines only
  BcrPlan bcr;                    // block cyclic reduction in place of multigrid (bcr.K > 0)
};
template <class Real>
void launch_bicg_init(const DevPtrs& d, cudaStream_t s);
template <class Real>
void launch_bicg_iter(const DevPtrs& d, const SolvePlan& plan, cudaStream_t s);
template <class Real>
cudaError_t set_poisson_smem(const SolvePlan& plan);
template <class Real>
void launch_line_factor(const DevPtrs& d, int level, int dir, int lines, int kmax, cudaStream_t s);
__host__ __device__ constexpr int line_fac_stride(int K) { return 5 * 32 * K + 13 * 32 + 2; }
__host__ __device__ constexpr int line_buf_len(int K) { return 32 * K + line_fac_stride(K); }
void launch_bicg_check(const DevPtrs& d, cudaGraphConditionalHandle h, int use_handle, cudaStream_t s);
// One cooperative launch for the whole solve (all Krylov iterations, all levels).
template <class Real>
cudaError_t launch_solve_coop(const DevPtrs& d, const SolvePlan& plan, int blocks, cudaStream_t s);
template <class Real>
int coop_blocks(const SolvePlan& plan, int sms);
// Dense inverse of an n x n FP64 matrix on the GPU (Gauss-Jordan, partial
// pivoting, one cooperative launch); work: n x 2n doubles, a[n][n] row-major
// on entry; out: Real[n][n]; cnt: the launch's grid-barrier counter (zeroed
// here); a barrier wait beyond wait_ns sets kErrTimeout in *err.
template <class Real>
cudaError_t launch_dense_inverse(double* work, double* fbuf, int n, Real* out, unsigned long long* cnt, int32_t* err,
                                 unsigned long long wait_ns, cudaStream_t s);
void launch_finish_injection(const DevPtrs& d, int pop, cudaStream_t s);

// Block cyclic reduction solve (bcr.cu): iterative refinement with an FP64
// residual and the FP32 reduction as the correction, one cooperative launch.
constexpr int kBcrRho = 1;     // form rho, the guess and b inside the solve
constexpr int kBcrFields = 2;  // node gradients and surface quantities after the solve
// only >= 0: solve that instance alone (its b and |b|^2 partials from the caller)
cudaError_t launch_solve_bcr(const DevPtrs& d, const SolvePlan& plan, int blocks, int mode, int only, cudaStream_t s);
// Several right-hand sides of the same systems in one launch (they share the
// blocks): the solution of system r of instance k is x[r] + node_off (initial
// guess on entry), its right-hand side b[r] + node_off, its |b|^2 partials in
// reduction slot slot[r]; n * n_inst <= kCoopMaxInst.
constexpr int kBcrMaxRhs = 3;
struct BcrRhs {
  int n;
  int slot[kBcrMaxRhs];
  double* x[kBcrMaxRhs];
  const double* b[kBcrMaxRhs];
};
cudaError_t launch_solve_bcr_rhs(const DevPtrs& d, const SolvePlan& plan, int blocks, const BcrRhs& rhs, cudaStream_t s);
// CTAs of the solve (0: not co-residable); sets each instance's staging flag
// and tail chunk, and the kernel's shared memory (plan.bcr.smem, plan.bcr.dyn).
int bcr_configure(SolvePlan& plan, BcrInst* inst, int n_inst, int sms);
const void* bcr_kernel(const SolvePlan& plan);  // the solve kernel (to find its graph node)
// blocks CTAs (all resident) wait at a barrier that never completes, each
// for d.wait_ns; d.bar must point at a zeroed counter of its own.
void launch_wait_check(const DevPtrs& d, int blocks, cudaStream_t s);

// sensitivity window (tangent.cu)
template <class Real>
void launch_tan_deposit(const DevPtrs& d, const TanPtrs& t, int grid, int max_n2, cudaStream_t s);
template <class Real>
void launch_tan_push(const DevPtrs& d, const TanPtrs& t, int grid, cudaStream_t s);
template <class Real>
void launch_tan_inject(const DevPtrs& d, const TanPtrs& t, long long max_inj, cudaStream_t s);
void launch_tan_rho(const DevPtrs& d, const TanPtrs& t, cudaStream_t s);
// direct = 0: b into DevPtrs::b (|b|^2 partials in slot 0) and the guess into
// DevPtrs::phi; direct = 1: b into TanPtrs::bt[p] (partials in slot
// kTanSlot + p), the guess stays in TanPtrs::dphi[p].
constexpr int kTanSlot = 5;
void launch_tan_b(const DevPtrs& d, const TanPtrs& t, int p, int direct, cudaStream_t s);
// direct = 0: dphi[p] = DevPtrs::phi inside, Dirichlet values on the
// boundary rows; direct = 1: the boundary rows only.
void launch_tan_store(const DevPtrs& d, const TanPtrs& t, int p, int direct, cudaStream_t s);
void launch_tan_surface(const DevPtrs& d, const TanPtrs& t, cudaStream_t s);
void launch_tan_step_end(const DevPtrs& d, const TanPtrs& t, cudaStream_t s);

// reverse sweep (adjoint.cu)
template <class Real>
void launch_adj_fwd_push(const DevPtrs& d, const AdjPtrs& a, int k, cudaStream_t s);
template <class Real>
void launch_adj_fwd_inject(const DevPtrs& d, const AdjPtrs& a, const TanPtrs& t, int k, long long max_inj,
                           cudaStream_t s);
template <class Real>
void launch_adj_rev_inject(const DevPtrs& d, const AdjPtrs& a, const TanPtrs& t, int k, long long max_inj,
                           cudaStream_t s);
template <class Real>
void launch_adj_rev_push(const DevPtrs& d, const AdjPtrs& a, const TanPtrs& t, int k, cudaStream_t s);
template <class Real>
void launch_adj_rev_deposit(const DevPtrs& d, const AdjPtrs& a, int k, cudaStream_t s);
void launch_adj_values(const DevPtrs& d, const AdjPtrs& a, cudaStream_t s);
void launch_adj_surface(const DevPtrs& d, const AdjPtrs& a, const TanPtrs& t, int k, cudaStream_t s);
void launch_adj_gradT(const DevPtrs& d, const AdjPtrs& a, cudaStream_t s);
void launch_adj_to_unknowns(const DevPtrs& d, const AdjPtrs& a, cudaStream_t s);
// the transposed sweeps over one tree level's fronts [f0, f1) of the instance
// whose unknowns start at unk0 (smem_doubles: its largest s + u)
void launch_adj_ndT(const AdjPtrs& a, int f0, int f1, long long unk0, int smem_doubles, bool forward, cudaStream_t s);
void launch_adj_after_solve(const DevPtrs& d, const AdjPtrs& a, const TanPtrs& t, int k, cudaStream_t s);
const void* adj_ndT_kernel();  // the transposed-sweep kernel (its shared-memory limit is raised at set-up)

}  // namespace apic
