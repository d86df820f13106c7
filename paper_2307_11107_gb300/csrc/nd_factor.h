// Nested-dissection factorisation of the Poisson correction system (Eqs. 6-7
// discretised on the node grid), formed once on the host in FP64 and stored
// as dense FP32 front matrices for the GPU solve (the nested-dissection
// tasks of bcr.cu's cooperative solve kernel).  Host-only C++.
//
// Unknowns: the nodes of rows i = 1..M (M = n1 - 1) of N = n2 + 1 nodes,
// u = (i - 1) N + j.  Row u couples to (i + di, j + dj), di, dj in {-1, 0, 1},
// and, on the pole rows j = 0 and j = N - 1, to (i, 2) and (i, N - 3) (the
// one-sided x2 derivative of the pole rows): the 11 stencil slots of the
// library (st_slot, kStPole).
//
// Ordering: the unknown rectangle is cut recursively by a row or a column of
// nodes (a separator: the 9-point couplings do not cross a full line, and a
// column cut is never placed at j = 1 or j = N - 2, which the pole couplings
// would jump) until the pieces hold at most `leaf` nodes.  Each cut is a
// front: its separator S (the line) and its update set U (the nodes outside
// its rectangle coupled to it, all on the separators of enclosing cuts).
// Eliminating the fronts from the leaves up is an LU factorisation of the
// system in this order (no pivoting across fronts; Gauss-Jordan with
// partial pivoting inside F_SS).  With F the front's assembled matrix,
//   forward (leaves first):  v_S = b_S + children's W at S, v_U = children's W at U,
//                            z_S = F_SS^-1 v_S,  W = v_U - (F_US F_SS^-1) v_S
//   backward (root first):   x_S = z_S - (F_SS^-1 F_SU) x_U
// so both sweeps are dense matrix-vector products, one tree level at a time.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace apic {

struct NdFront {
  int level;      // depth below the root (root 0)
  int s, u;       // separator and update-set sizes
  int sp, up;     // row strides of its matrices (s, u rounded up to 4 floats)
  int child[2];   // children (-1: none)
  int parent;     // -1 for the root
  int pad;
  int64_t S, U;   // first entry of its separator / update set in NdFactor::idx (unknown indices)
  int64_t G;      // first entry of its gather table in NdFactor::gather: 2 (s + u) ints, for every position of
                  // [S; U] the index into child 0's and child 1's update vectors (-1: none)
  int64_t W;      // first float of its update vector (u entries) in the update buffer
  int64_t FM;     // first float of [F_SS^-1; F_US F_SS^-1]: (s + u) rows of sp floats, row-major
  int64_t NB;     // first float of F_SS^-1 F_SU: s rows of up floats, row-major
};

struct NdFactor {
  int M = 0, N = 0, depth = 0;
  std::vector<NdFront> fronts;                 // children before parents
  std::vector<std::vector<int>> by_level;      // front indices per level (0 = root)
  std::vector<int32_t> idx, gather;
  int64_t w_total = 0, fm_total = 0, nb_total = 0;
  std::vector<float> fm, nb;                   // FP32 front matrices (the GPU's copy)
  std::vector<double> fm64, nb64;              // FP64 copies (kept only when requested)
  int max_s = 0, max_u = 0;
};

// coef(i, j, slot): coefficient of the slot's neighbour in the row of node
// (i, j) (i = 1..M, j = 0..N-1); slots 0..8 are 3 (di + 1) + (dj + 1), slot 9
// the pole reach (j = 0 -> 2, j = N-1 -> N-3), slot 10 unused.  Neighbours on
// the Dirichlet rows (i = 0, M + 1) are not unknowns and are ignored.
using NdCoef = double (*)(const void* ctx, int i, int j, int slot);

// Builds the ordering and the factorisation with `threads` host threads.
// keep64: keep the FP64 matrices too (host solve in FP64).  Returns false
// (with a reason) for a singular front or sizes beyond the limits.
bool nd_build(int M, int N, NdCoef coef, const void* ctx, int leaf, int threads, bool keep64, NdFactor& f,
              std::string& why);

// Host version of the GPU's two sweeps: e = A^-1 r (r, e: M N unknowns), with
// the FP32 matrices (or the FP64 ones when kept and fp64 is set).
void nd_solve_host(const NdFactor& f, const double* r, double* e, bool fp64);

// ---- device tables (what the GPU's nested-dissection tasks read) ----
// A task of one tree level: rows [r0, r0 + n) of the large front `front`
// (warp = 0, the whole CTA), the n small fronts from `front` (warp = 1, one
// warp each), or the n tiny fronts from `front` (warp = 2, four per warp, one
// per 8-lane group).  Same layout as CUDA's int4.
struct NdTask {
  int front, r0, n, warp;
};
constexpr int kNdTinyS = 16;  // tiny fronts: separator and update set within these sizes
constexpr int kNdTinyU = 48;
// Fronts of a batch's instances, sorted by level within each instance, with
// offsets made global: S, U into idx; G into gather; W into one right-hand
// side's update vectors; FM, NB into the batch's matrix buffer.
struct NdUpload {
  std::vector<NdFront> fronts;
  std::vector<int32_t> idx, gather;
  std::vector<NdTask> tasks;
};
// Task ranges of one instance: forward tasks of level l are tasks
// [ft[l], ft[l + 1]), backward ones [bt[l], bt[l + 1]).
struct NdLevels {
  std::vector<int32_t> ft, bt;
};

// Appends instance f to `up` with its matrices at float `mat` of the matrix
// buffer (FM first, then NB) and its update vectors at float `wb`.  Fronts
// with s > warp_s, u > warp_u or more than warp_floats matrix floats in a
// sweep are large in that sweep (row chunks of at most task_floats matrix
// floats and task_rows rows, each a task of a whole worker); the small
// fronts of a level are
// spread over `ctas` tasks (at most task_fronts each, one per warp), so that a
// level keeps every CTA busy, the tiny ones four to a warp when there are at
// least four per CTA.  A task's matrix rows are one contiguous range of at
// most stage_floats floats (requires task_floats <= stage_floats and
// warp_floats task_fronts <= stage_floats).  In `up`, gather entries are
// absolute offsets into one right-hand side's update vectors (-1: none).
// Returns the floats of shared memory a large front's vector needs.
int nd_layout(const NdFactor& f, int64_t mat, int64_t wb, int warp_s, int warp_u, int warp_floats, int task_floats,
              int task_rows, int task_fronts, int stage_floats, int ctas, NdUpload& up, NdLevels& lv);

// The sweeps as the device runs them, task by task from the tables above, for
// one instance of `up` (task ranges lv, tree depth `depth`; its matrices in
// matbuf at the offsets its fronts hold): e = A^-1 r with the FP32 matrices
// and FP32 vectors, w the update vectors (one right-hand side's range).
void nd_solve_tables(const NdUpload& up, const NdLevels& lv, int depth, const std::vector<float>& matbuf, int N,
                     const float* r, float* e, std::vector<float>& w);

}  // namespace apic
