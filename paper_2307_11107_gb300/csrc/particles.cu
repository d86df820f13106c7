// Particle kernels of the APIC step (arXiv:2307.11107, Secs. 1-2): volume
// load, surface injection (Eq. 4), field gather (Eq. 10) + Boris push (Eq. 9)
// + absorption tallies + escape, and charge weighing (Eq. 5) into 64-bit
// fixed-point node accumulators.
//
// This file is compiled once per particle precision: -DAPIC_REAL=double (with
// -fmad=false, the parity build) and -DAPIC_REAL=float.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstdlib>

#include <cstdint>

#include "apic_internal.h"
#include "geom.cuh"

#ifndef APIC_REAL
#error "compile with -DAPIC_REAL=float or -DAPIC_REAL=double"
#endif

namespace apic {
namespace {

#include "particle_common.cuh"
#include "bulk_copy.cuh"

constexpr unsigned kFull = 0xffffffffu;
constexpr int kPushItems = 8;    // particles per thread per chunk
constexpr int kFlushChunks = 31;  // chunks (of 2048 particles) between window flushes at most
// the vector push: particles per thread per chunk, 16 (4096 per chunk) or 32
// (8192: fewer barriers per particle, coarser load balance); a window is
// flushed before a cell's packed moments could hold 2^16 particles
constexpr int kPush4ItemsMax = 32;
constexpr int kWinRows = 8;      // node rows of the initial deposit's shared-memory window
constexpr int kPushWinRows = 16; // node rows of the push's shared-memory deposit window at most
constexpr int kWinMaxN2 = 513;   // widest grid row the window holds (larger grids deposit globally)
constexpr int kInjRows = 3;      // node rows of the injection window (the last two cell rows)
constexpr int kInjMaxN2 = 512;   // widest grid (cells in x2) the injection window holds

struct W4 {
  unsigned long long w00, w10, w01, w11;
};

// Fixed-point cloud-in-cell weights.  FP64: each weight rounded to F bits.
// FP32: fractions quantised to F/2 bits, weights as exact integer products
// (their sum is exactly 2^F: charge is conserved to the last bit).
__device__ __forceinline__ W4 weights(const Cell& c, int F) {
  W4 w;
  if (kF64) {
    double sc = ldexp(1.0, F);
    double g1 = 1.0 - (double)c.f1, g2 = 1.0 - (double)c.f2;
    w.w00 = (unsigned long long)__double2ll_rn(g1 * g2 * sc);
    w.w10 = (unsigned long long)__double2ll_rn((double)c.f1 * g2 * sc);
    w.w01 = (unsigned long long)__double2ll_rn(g1 * (double)c.f2 * sc);
    w.w11 = (unsigned long long)__double2ll_rn((double)c.f1 * (double)c.f2 * sc);
  } else {
    int b = F >> 1;
    unsigned one = 1u << b;
    unsigned q1 = (unsigned)((float)c.f1 * (float)one + 0.5f), q2 = (unsigned)((float)c.f2 * (float)one + 0.5f);
    q1 = q1 > one ? one : q1;
    q2 = q2 > one ? one : q2;
    w.w00 = (unsigned long long)(one - q1) * (one - q2);
    w.w10 = (unsigned long long)q1 * (one - q2);
    w.w01 = (unsigned long long)(one - q1) * q2;
    w.w11 = (unsigned long long)q1 * q2;
  }
  return w;
}

// Runs of consecutive lanes holding the same key (invalid lanes are runs of
// their own): start lane, length and rank of every lane in its run.
struct Run {
  int start, len, rank;
};

__device__ __forceinline__ Run warp_runs(long long key, bool valid) {
  const int lane = threadIdx.x & 31;
  long long kp = __shfl_up_sync(kFull, key, 1);
  int vp = __shfl_up_sync(kFull, (int)valid, 1);
  bool head = lane == 0 || !valid || !vp || kp != key;
  unsigned hm = __ballot_sync(kFull, head);
  unsigned upto = hm & ((2u << lane) - 1u);
  Run r;
  r.start = 31 - __clz(upto);
  unsigned after = hm & ~((2u << lane) - 1u);
  int next = after ? __ffs(after) - 1 : 32;
  r.len = next - r.start;
  r.rank = lane - r.start;
  return r;
}

// Sum of v over the lanes of each run, held by the run's last lane.
__device__ __forceinline__ unsigned long long run_sum(unsigned long long v, const Run& r) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    unsigned long long up = __shfl_up_sync(kFull, v, o);
    if (lane - o >= r.start) v += up;
  }
  return v;
}

// Accumulation target of one CTA: a shared-memory window of node rows
// [row0, row0 + rows) of one population (all columns), flushed to the global
// accumulator once per chunk; corners outside it go straight to global memory.
struct Window {
  unsigned long long* s;  // shared [rows * N2]
  unsigned long long* g;  // global accumulator of the population (node 0)
  int row0, rows, N2;
};

__device__ __forceinline__ void win_add(const Window& W, int i, int j, unsigned long long v) {
  if (!v) return;
  int rr = i - W.row0;
  if (rr >= 0 && rr < W.rows) atomicAdd(W.s + rr * W.N2 + j, v);
  else atomicAdd(W.g + (long long)i * W.N2 + j, v);
}

__device__ __forceinline__ void add4(const Window& W, int i, int j, unsigned long long w00, unsigned long long w10,
                                     unsigned long long w01, unsigned long long w11) {
  win_add(W, i, j, w00);
  win_add(W, i + 1, j, w10);
  win_add(W, i, j + 1, w01);
  win_add(W, i + 1, j + 1, w11);
}

// Deposit of one lane's four corner weights into the window (or global
// memory).  Integer addition makes the result independent of the order.
__device__ __forceinline__ void deposit_lane(const Window& W, int ci, int cj, const W4& w, bool active) {
  if (active) add4(W, ci, cj, w.w00, w.w10, w.w01, w.w11);
}

// FP32 deposit through cell moments.  With fractions quantised to b = 16
// bits (S = 2^16, rounded to nearest; an FP32 position resolves about 2^-16
// of a cell anyway) the four corner weights of a particle are (S-q1)(S-q2),
// q1(S-q2), (S-q1)q2, q1 q2: linear in the moments (1, q1, q2, q1 q2), so a
// cell accumulates only those, packed in two words (q1 << 32 | q2, and
// q1 q2 + 2^48), and the corner weights of all its particles follow exactly
// from the sums at the flush.  For at most 65535 particles in a cell between
// flushes the fields cannot carry into each other (sum q2 < 2^32, sum q1 q2
// < 2^48, count < 2^16): kFlushChunks chunks of 2048 particles.
// Cell (rr, cj) of an FP32 window: its packed sums (q1 << 32 | q2) at word
// win_a(rr, cj) and (count << 48) + sum q1 q2 at win_a + win_m: the two words
// in separate planes of rows x win_n2 words, so that a warp's random cells
// spread over twice as many banks as with the pair side by side (the
// 1024 x 512 push: 1.335 against 1.391 ms).
__device__ __forceinline__ int win_a(int rr, int cj, int n2) { return rr * n2 + cj; }
__device__ __forceinline__ int win_m(int plane) { return plane; }

struct CellWin {
  unsigned long long* s;  // shared [rows * n2 * 2]
  unsigned long long* g;  // global node accumulator of the population (node 0)
  int row0, rows, n2, N2;
  int plane;  // words of one plane (win_rows x win_n2)
};

__device__ __forceinline__ void corner_weights(unsigned long long a, unsigned long long m, unsigned S,
                                               unsigned long long w[4]) {
  const unsigned long long n = m >> 48, s12 = m & ((1ull << 48) - 1ull), s1 = a >> 32, s2 = a & 0xffffffffull;
  const unsigned long long SS = (unsigned long long)S * S;
  w[0] = n * SS - (unsigned long long)S * (s1 + s2) + s12;
  w[1] = (unsigned long long)S * s1 - s12;
  w[2] = (unsigned long long)S * s2 - s12;
  w[3] = s12;
}

__device__ __forceinline__ void cell_add(const CellWin& W, int ci, int cj, unsigned long long a, unsigned long long m,
                                         unsigned S) {
  const int rr = ci - W.row0;
  if (rr >= 0 && rr < W.rows) {
    // the two 64-bit moments by 32-bit shared-memory atomics (64-bit ones
    // measured about three times as costly): the halves of `a` never carry
    // (sum q1 and sum q2 stay below 2^32 between flushes), the low half of `m`
    // passes its carry to the high half
    unsigned long long* c = W.s + win_a(rr, cj, W.n2);
    unsigned* a32 = (unsigned*)c;
    unsigned* m32 = (unsigned*)(c + win_m(W.plane));
    atomicAdd(a32, (unsigned)a);
    atomicAdd(a32 + 1, (unsigned)(a >> 32));
    const unsigned lo = (unsigned)m, old = atomicAdd(m32, lo);
    atomicAdd(m32 + 1, (unsigned)(m >> 32) + (old + lo < old ? 1u : 0u));
  } else {
    unsigned long long w[4];
    corner_weights(a, m, S, w);
    unsigned long long* g = W.g + (long long)ci * W.N2 + cj;
    if (w[0]) atomicAdd(g, w[0]);
    if (w[1]) atomicAdd(g + W.N2, w[1]);
    if (w[2]) atomicAdd(g + 1, w[2]);
    if (w[3]) atomicAdd(g + W.N2 + 1, w[3]);
  }
}

// One particle per lane.  (Summing a warp's moments first when all its lanes
// share one cell measured slower on row-sorted particles: the warp-wide test
// costs more than the rare shared atomics it saves.)
__device__ __forceinline__ void deposit_moments(const CellWin& W, int key, int ci, int cj, unsigned q1, unsigned q2,
                                                int b, bool active) {
  const unsigned S = 1u << b;
  const unsigned long long p12 = (unsigned long long)q1 * q2;
  (void)key;
  if (active) cell_add(W, ci, cj, ((unsigned long long)q1 << 32) | q2, p12 + (1ull << 48), S);
}

__device__ __forceinline__ long long dep_key(const Inst& I, const Pop& P, const Cell& c) {
  return P.acc_off + (long long)c.i * I.N2 + c.j;
}

// Per-population constants of the push, staged in shared memory.
struct PushConst {
  Real al, h1, h2, x1_out, dt, B, h;  // h = q dt / (2 m)
  Real ih1, ih2, tz, sz;              // 1/h1, 1/h2, Boris rotation factors (constant per population)
  int n1, n2, N2, fbits;
  long long node_off, acc_off;
};

__device__ __forceinline__ Cell locate_c(const PushConst& C, Real x1, Real x2) {
  Real u1 = (x1 + Real(1)) / C.h1;
  Real u2 = (x2 + Real(1)) / C.h2;
  Cell c;
  c.i = (int)floor(u1);
  c.j = (int)floor(u2);
  c.i = c.i < 0 ? 0 : (c.i > C.n1 - 1 ? C.n1 - 1 : c.i);
  c.j = c.j < 0 ? 0 : (c.j > C.n2 - 1 ? C.n2 - 1 : c.j);
  c.f1 = u1 - (Real)c.i;
  c.f2 = u2 - (Real)c.j;
  c.f1 = c.f1 < Real(0) ? Real(0) : (c.f1 > Real(1) ? Real(1) : c.f1);
  c.f2 = c.f2 < Real(0) ? Real(0) : (c.f2 > Real(1) ? Real(1) : c.f2);
  return c;
}

// One full particle update for slot t of the batch (Sec. 2, Eqs. 8-10, 9).
// The CTA works on chunks of kPushItems x blockDim consecutive slots of one
// population (sorted by cell, so a chunk covers few grid rows) and deposits
// into a shared-memory window of win_rows (<= kWinRows) node rows that is flushed to the
// global accumulator after each chunk.
#ifndef APIC_PUSH_UNROLL
#define APIC_PUSH_UNROLL 2
#endif
constexpr int kPushUnroll = APIC_PUSH_UNROLL;  // items of the chunk loop unrolled
#ifndef APIC_PUSH_MIN_BLOCKS
// FP32: 64 registers, four CTAs of 256 threads per SM; FP64 (parity build): two
#define APIC_PUSH_MIN_BLOCKS (sizeof(APIC_REAL) == 4 ? 4 : 2)
#endif
// kChord: some instance absorbs grazing orbits (APIC_CHORD_ABSORB); the
// instantiation without it carries no trace of the test.
template <bool kChord>
__global__ void __launch_bounds__(256, APIC_PUSH_MIN_BLOCKS) k_push(DevPtrs d, int win_n2, int win_rows, int group) {
  // dynamic shared memory: the deposit window, then the chunk prefix over the
  // populations and their constants (sized by the batch, so that a small
  // batch leaves more of the SM's memory to L1 for the field gather)
  extern __shared__ unsigned long long s_win[];
  const int win_words = kF64 ? win_rows * (win_n2 + 1) : 2 * win_rows * win_n2;
  const int plane = win_rows * win_n2;  // FP32 window: words of one plane
  long long* s_pre = (long long*)(s_win + win_words);
  PushConst* s_pc = (PushConst*)(s_pre + d.n_pop + 1);
  __shared__ int s_row0, s_wpop, s_nsince, s_newrow0, s_flush, s_gi;
  __shared__ unsigned s_rowmask;  // FP32 window: cell rows that received moments in this chunk
  const long long CH = (long long)kPushItems * blockDim.x;
  if (threadIdx.x == 0) {
    long long a = 0;
    for (int p = 0; p < d.n_pop; ++p) {
      s_pre[p] = a;
      a += (d.ps[p].n + CH - 1) / CH;
    }
    s_pre[d.n_pop] = a;
  }
  for (int p = threadIdx.x; p < d.n_pop; p += blockDim.x) {
    const Pop& P = d.pop[p];
    const Inst& I = d.inst[P.inst];
    PushConst C;
    C.al = (Real)I.alpha;
    C.h1 = (Real)I.h1;
    C.h2 = (Real)I.h2;
    C.x1_out = (Real)I.x1_out;
    C.dt = (Real)I.dt;
    C.B = (Real)I.B;
    C.h = Real(0.5) * (Real)(P.q / P.m) * (Real)I.dt;
    C.ih1 = (Real)(1.0 / I.h1);
    C.ih2 = (Real)(1.0 / I.h2);
    C.tz = C.h * (-(Real)I.B);
    C.sz = Real(2) * C.tz / (Real(1) + C.tz * C.tz);
    C.n1 = I.n1;
    C.n2 = I.n2;
    C.N2 = I.N2;
    C.fbits = P.fbits;
    C.node_off = I.node_off;
    C.acc_off = P.acc_off;
    s_pc[p] = C;
  }
  for (int k = threadIdx.x; k < win_words; k += blockDim.x) s_win[k] = 0ull;
  __syncthreads();
  const long long total_chunks = s_pre[d.n_pop];
  Real* X1 = (Real*)d.x1;
  Real* X2 = (Real*)d.x2;
  Real* VR = (Real*)d.vR;
  Real* VZ = (Real*)d.vZ;
  Real* VT = (Real*)d.vT;
  const Real2* G = (const Real2*)d.G;
  // Flush of the window (population wp, node rows from row0) to the global
  // accumulator, and its clearing.
  auto flush = [&](int wp, int row0) {
    const PushConst& Cw = s_pc[wp];
    const int rows = Cw.n2 <= win_n2 ? win_rows : 0;
    unsigned long long* g = d.acc + Cw.acc_off;
    if (kF64) {
      for (int e = threadIdx.x; e < rows * Cw.N2; e += blockDim.x) {
        unsigned long long v = s_win[e];
        if (v) {
          atomicAdd(g + (long long)(row0 + e / Cw.N2) * Cw.N2 + e % Cw.N2, v);
          s_win[e] = 0ull;
        }
      }
    } else {
      // node (ni, nj) of rows row0..row0+rows gathers w00 of cell (ni, nj),
      // w10 of (ni-1, nj), w01 of (ni, nj-1) and w11 of (ni-1, nj-1)
      // (only the node rows next to the cell rows that received moments)
      const unsigned S = 1u << (Cw.fbits >> 1);
      const unsigned cm = s_rowmask;
      const unsigned nm = cm | (cm << 1);  // node rows rr with cell row rr or rr - 1 in use
      const int nrows = __popc(nm);
      for (int e = threadIdx.x; e < nrows * Cw.N2; e += blockDim.x) {
        const int q = e / Cw.N2, nj = e - q * Cw.N2;
        unsigned mm = nm;
        for (int z = 0; z < q; ++z) mm &= mm - 1u;
        const int rr = __ffs(mm) - 1;  // the q-th node row in use
        unsigned long long v = 0, w[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const int cr = rr - (t & 1), cj = nj - (t >> 1);
          if (cr < 0 || cr >= rows || !((cm >> cr) & 1u) || cj < 0 || cj >= Cw.n2) continue;
          const unsigned long long* c = s_win + win_a(cr, cj, Cw.n2);
          if (c[win_m(plane)] == 0ull) continue;
          corner_weights(c[0], c[win_m(plane)], S, w);
          v += w[t];  // t = 0: w00 (own cell), 1: w10 (cell below in x1), 2: w01, 3: w11
        }
        if (v) atomicAdd(g + (long long)(row0 + rr) * Cw.N2 + nj, v);
      }
      __syncthreads();
      const int crows = __popc(cm);
      for (int e = threadIdx.x; e < 2 * crows * Cw.n2; e += blockDim.x) {
        const int q = e / (2 * Cw.n2), o = e - q * 2 * Cw.n2;
        unsigned mm = cm;
        for (int z = 0; z < q; ++z) mm &= mm - 1u;
        const int rz = __ffs(mm) - 1;
        s_win[o < Cw.n2 ? win_a(rz, o, Cw.n2) : win_a(rz, o - Cw.n2, Cw.n2) + win_m(plane)] = 0ull;
      }
    }
    __syncthreads();
  };
  // This CTA's chunks are a contiguous range of the sorted particles (few
  // grid rows), deposited into one window that is flushed only when a chunk's
  // rows or population leave it, or after kFlushChunks chunks: the global
  // atomics of the flushes, which all CTAs working on one grid row send to
  // the same addresses, are what the window saves.
  // groups of `group` consecutive chunks, taken in order from a counter that
  // is cleared before each launch: the CTAs balance themselves, and the CTAs
  // at work read neighbouring memory
  const int nch = (int)total_chunks;  // chunks of 2048 particles: far below 2^31
  const int GS = group > 0 ? group : 1;
  const int ngroups = (nch + GS - 1) / GS;
  if (threadIdx.x == 0) {
    s_wpop = -1;
    s_nsince = 0;
    s_rowmask = 0u;
  }
  __syncthreads();
  for (int q = 0;; ++q) {
   if (q % GS == 0) {
     // every warp has read the previous group's index (chunks past the last
     // one are skipped without a barrier, so warps may drift apart there)
     __syncthreads();
     if (threadIdx.x == 0) s_gi = (int)atomicAdd((unsigned long long*)(d.cnt + 1), 1ull);
     __syncthreads();
   }
   const int gi = s_gi;
   if (gi >= ngroups) break;
   const long long chunk = (long long)gi * GS + q % GS;
   if (chunk >= nch) continue;
   const int pop = find_pop(s_pre, d.n_pop, chunk);
   // by value: the constants stay in registers instead of being reloaded from
   // shared memory around every window atomic
   const PushConst C = s_pc[pop];
   const long long npop = d.ps[pop].n, pbase = d.pop[pop].base;
   const long long c0 = (chunk - s_pre[pop]) * CH;
   if (threadIdx.x == 0) {
     int row = 0;
     for (int q = 0; q < 64 && c0 + q < npop; ++q) {
       Real xq = X1[pbase + c0 + q];
       if (xq < Real(0)) {
         row = (int)floor((double)((xq + Real(1)) * C.ih1));
         break;
       }
     }
     const int r0 = row > 0 ? row - 1 : 0;
     const int rows = C.n2 <= win_n2 ? win_rows : 0;
     // keep the window while this chunk's first rows lie inside it
     const bool keep = s_wpop == pop && s_nsince < kFlushChunks && r0 >= s_row0 && r0 + 2 < s_row0 + rows;
     s_flush = s_wpop >= 0 && !keep;
     s_newrow0 = keep ? s_row0 : r0;
   }
   __syncthreads();
   if (s_flush) flush(s_wpop, s_row0);
   if (threadIdx.x == 0) {
     if (s_row0 != s_newrow0 || s_wpop != pop || s_flush) {
       s_row0 = s_newrow0;
       s_wpop = pop;
       s_rowmask = 0u;
       s_nsince = 0;
     }
     s_nsince += 1;
   }
   __syncthreads();
   Window W;
   W.s = s_win;
   W.g = d.acc + C.acc_off;
   W.row0 = s_row0;
   W.N2 = C.N2;
   W.rows = C.n2 <= win_n2 ? win_rows : 0;
   CellWin CW;
   CW.s = s_win;
   CW.plane = plane;
   CW.g = W.g;
   CW.row0 = W.row0;
   CW.rows = W.rows;
   CW.n2 = C.n2;
   CW.N2 = C.N2;
   // this thread's items sit at 32-bit offsets it * blockDim.x from per-chunk
   // pointers; the state of the next item is loaded while the current one is pushed
   const long long t0 = pbase + c0 + threadIdx.x;
   const long long left = npop - c0 - threadIdx.x;
   const int nleft = left > CH ? (int)CH : (int)left;  // offsets below nleft are in the population
   const Real2* Gi = G + C.node_off;
   Real nx1 = Real(2), nx2 = Real(0), nvR = Real(0), nvZ = Real(0), nvT = Real(0);
   auto fetch = [&](int it) {
     const int o = it * (int)blockDim.x;
     if (o < nleft) {
       const long long q = t0 + o;
       nx1 = X1[q];
       nx2 = X2[q];
       nvR = VR[q];
       nvZ = VZ[q];
       nvT = VT[q];
     } else {
       nx1 = Real(2);
     }
   };
   fetch(0);
#pragma unroll kPushUnroll
   for (int it = 0; it < kPushItems; ++it) {
    const int o = it * (int)blockDim.x;
    const bool active = o < nleft;
    const Real x1 = nx1, cx2 = nx2, cvR = nvR, cvZ = nvZ, cvT = nvT;
    if (it + 1 < kPushItems) fetch(it + 1);
    bool alive = active && x1 < Real(0);
    int fate = 0;  // 1 absorbed, 2 escaped
    int key = -1, di = 0, dj = 0;
    W4 w = {0, 0, 0, 0};
    unsigned q1 = 0, q2 = 0;
    if (alive && !kF64) {
      // FP32: reciprocals and rsqrt instead of divisions; the grain test
      // r < (1 + sqrt(1 + 4 alpha x2))/2 is taken on squares.
      float x2 = cx2, vR = cvR, vZ = cvZ, vT = cvT;
      const float al = C.al, dt = C.dt;
      float x1f = (float)x1;
      float disc = 1.0f - 4.0f * al * x1f * x2;
      float ir = __fdividef(-2.0f * x1f, 1.0f + sqrtf(disc));  // 1/r (Eq. 3)
      float r = __fdividef(1.0f, ir);
      float s2 = (1.0f - x2) * (1.0f + x2);
      float sn = sqrtf(s2);
      float R = r * sn, Z = r * x2;
      float u1 = (x1f + 1.0f) * C.ih1, u2 = (x2 + 1.0f) * C.ih2;
      int ci = min(max((int)floorf(u1), 0), C.n1 - 1), cj = min(max((int)floorf(u2), 0), C.n2 - 1);
      float f1 = fminf(fmaxf(u1 - (float)ci, 0.0f), 1.0f), f2 = fminf(fmaxf(u2 - (float)cj, 0.0f), 1.0f);
      const int n00 = ci * C.N2 + cj;
      Real2 a00 = Gi[n00], a10 = Gi[n00 + C.N2], a01 = Gi[n00 + 1], a11 = Gi[n00 + C.N2 + 1];
      float g1 = (1.0f - f2) * ((1.0f - f1) * a00.x + f1 * a10.x) + f2 * ((1.0f - f1) * a01.x + f1 * a11.x);
      float g2 = (1.0f - f2) * ((1.0f - f1) * a00.y + f1 * a10.y) + f2 * ((1.0f - f1) * a01.y + f1 * a11.y);
      float ir3 = ir * ir * ir;
      float x1R = sn * (r + 3.0f * al * x2) * ir3, x1Z = (r * x2 + al * (3.0f * x2 * x2 - 1.0f)) * ir3;
      float x2R = -x2 * sn * ir, x2Z = s2 * ir;
      float ER = -(x1R * g1 + x2R * g2), EZ = -(x1Z * g1 + x2Z * g2);
      float h = C.h, tz = C.tz, sz = C.sz;
      float vx = vR + h * ER, vy = vT, vz = vZ + h * EZ;
      float px_ = vx + vy * tz, py_ = vy - vx * tz;
      vx = vx + py_ * sz + h * ER;
      vy = vy - px_ * sz;
      vz = vz + h * EZ;
      float Xc = R + vx * dt, Yc = vy * dt, Zn = Z + vz * dt;
      float Rn2 = Xc * Xc + Yc * Yc;
      float cr = 1.0f, sr = 0.0f;
      if (Rn2 > 0.0f) {
        float iR = rsqrtf(Rn2);
        cr = Xc * iR;
        sr = Yc * iR;
      }
      float vRn = cr * vx + sr * vy, vTn = -sr * vx + cr * vy;
      float rn2 = Rn2 + Zn * Zn;
      float irn = rsqrtf(rn2);
      float rn = rn2 * irn;
      float x2n = Zn * irn;
      float tr = 2.0f * rn - 1.0f;
      bool hit = tr < 0.0f || tr * tr < 1.0f + 4.0f * al * x2n;
      float tau = dt;  // chord time up to a point inside the grain
      if (kChord && !hit && (d.inst[d.pop[pop].inst].flags & APIC_CHORD_ABSORB)) {
        const float se = chord_entry(al, R, Z, vx * dt, vy * dt, vz * dt);
        if (se > 0.0f) {
          hit = true;
          tau = dt * se;
        }
      }
      if (hit) {
        const Pop& P = d.pop[pop];
        absorb_tally(d, d.inst[P.inst], P, R, Z, vx, vz, vy, tau);
        X1[t0 + o] = Real(2);
        fate = 1;
      } else {
        float x1n = -irn * (1.0f + al * x2n * irn);
        if (x1n > C.x1_out) {
          X1[t0 + o] = Real(2);
          fate = 2;
        } else {
          X1[t0 + o] = x1n;
          X2[t0 + o] = x2n;
          VR[t0 + o] = vRn;
          VZ[t0 + o] = vz;
          VT[t0 + o] = vTn;
          float v1 = (x1n + 1.0f) * C.ih1, v2 = (x2n + 1.0f) * C.ih2;
          int ni = min(max((int)floorf(v1), 0), C.n1 - 1), nj = min(max((int)floorf(v2), 0), C.n2 - 1);
          float e1 = fminf(fmaxf(v1 - (float)ni, 0.0f), 1.0f), e2 = fminf(fmaxf(v2 - (float)nj, 0.0f), 1.0f);
          const float one = (float)(1u << (C.fbits >> 1));
          q1 = min((unsigned)(e1 * one + 0.5f), 1u << (C.fbits >> 1));
          q2 = min((unsigned)(e2 * one + 0.5f), 1u << (C.fbits >> 1));
          key = ni * C.N2 + nj;
          di = ni;
          dj = nj;
        }
      }
    } else if (alive) {
      Real x2 = cx2, vR = cvR, vZ = cvZ, vT = cvT;
      const Real al = C.al, dt = C.dt;
      Real r = radius(al, x1, x2);
      Real sn = sqrt((Real(1) - x2) * (Real(1) + x2));
      Real R = r * sn, Z = r * x2;
      // gather (Eq. 10): bilinear node gradients, analytic metric at the particle
      Cell c = locate_c(C, x1, x2);
      const int n00 = c.i * C.N2 + c.j;
      Real2 a00 = Gi[n00], a10 = Gi[n00 + C.N2], a01 = Gi[n00 + 1], a11 = Gi[n00 + C.N2 + 1];
      Real w00 = (Real(1) - c.f1) * (Real(1) - c.f2), w10 = c.f1 * (Real(1) - c.f2);
      Real w01 = (Real(1) - c.f1) * c.f2, w11 = c.f1 * c.f2;
      Real g1 = w00 * a00.x + w10 * a10.x + w01 * a01.x + w11 * a11.x;
      Real g2 = w00 * a00.y + w10 * a10.y + w01 * a01.y + w11 * a11.y;
      Metric<Real> m = metric(al, r, x2);
      Real ER = -(m.x1R * g1 + m.x2R * g2);
      Real EZ = -(m.x1Z * g1 + m.x2Z * g2);
      // Boris in the local frame (R-hat, Theta-hat, Z-hat); Eq. 9's Lorentz
      // terms are those of the field vector -B z-hat.
      Real h = C.h;
      Real vx = vR + h * ER, vy = vT, vz = vZ + h * EZ;
      Real tz = h * (-C.B);
      Real sz = Real(2) * tz / (Real(1) + tz * tz);
      Real px_ = vx + vy * tz, py_ = vy - vx * tz;
      vx = vx + py_ * sz;
      vy = vy - px_ * sz;
      vx = vx + h * ER;
      vz = vz + h * EZ;
      // straight chord, rotation back to the meridional half plane
      Real Xc = R + vx * dt, Yc = vy * dt, Zn = Z + vz * dt;
      Real Rn = sqrt(Xc * Xc + Yc * Yc);
      Real cr = Real(1), sr = Real(0);
      if (Rn > Real(0)) {
        cr = Xc / Rn;
        sr = Yc / Rn;
      }
      Real vRn = cr * vx + sr * vy, vTn = -sr * vx + cr * vy;
      Real rn = sqrt(Rn * Rn + Zn * Zn);
      Real x2n = Zn / rn;
      bool hit = rn < r_grain(al, x2n);
      Real tau = dt;  // chord time up to a point inside the grain
      if (kChord && !hit && (d.inst[d.pop[pop].inst].flags & APIC_CHORD_ABSORB)) {
        const Real se = chord_entry(al, R, Z, vx * dt, vy * dt, vz * dt);
        if (se > Real(0)) {
          hit = true;
          tau = dt * se;
        }
      }
      if (hit) {
        const Pop& P = d.pop[pop];
        absorb_tally(d, d.inst[P.inst], P, R, Z, vx, vz, vy, tau);
        X1[t0 + o] = Real(2);
        fate = 1;
      } else {
        Real x1n = x1_at(al, rn, x2n);
        if (x1n > C.x1_out) {
          X1[t0 + o] = Real(2);
          fate = 2;
        } else {
          X1[t0 + o] = x1n;
          X2[t0 + o] = x2n;
          VR[t0 + o] = vRn;
          VZ[t0 + o] = vz;
          VT[t0 + o] = vTn;
          Cell cn = locate_c(C, x1n, x2n);
          key = cn.i * C.N2 + cn.j;
          di = cn.i;
          dj = cn.j;
          w = weights(cn, C.fbits);
        }
      }
    }
    // counters and freed slots, one atomic per warp and outcome (every lane of
    // the chunk's warp belongs to the same population)
    {
      const unsigned lane = threadIdx.x & 31;
      const unsigned m_abs = __ballot_sync(kFull, fate == 1), m_gone = __ballot_sync(kFull, fate != 0);
      if (m_gone) {
        const int leader = __ffs(m_gone) - 1;
        long long h0 = 0;
        if ((int)lane == leader) {
          PopState& S = d.ps[pop];
          if (m_abs) atomicAdd((unsigned long long*)&S.absorbed, (unsigned long long)__popc(m_abs));
          if (m_gone & ~m_abs) atomicAdd((unsigned long long*)&S.escaped, (unsigned long long)__popc(m_gone & ~m_abs));
          h0 = (long long)atomicAdd((unsigned long long*)&S.n_holes, (unsigned long long)__popc(m_gone));
        }
        h0 = __shfl_sync(kFull, h0, leader);
        if (fate != 0)
          d.holes[d.pop[pop].base + h0 + __popc(m_gone & ((1u << lane) - 1u))] = (int32_t)(c0 + threadIdx.x + o);
      }
    }
    if (kF64) {
      deposit_lane(W, di, dj, w, key >= 0);
    } else {
      deposit_moments(CW, key, di, dj, q1, q2, C.fbits >> 1, key >= 0);
      const int rr = di - CW.row0;
      const unsigned rows_hit = __reduce_or_sync(kFull, (key >= 0 && rr >= 0 && rr < CW.rows) ? (1u << rr) : 0u);
      if ((threadIdx.x & 31) == 0 && rows_hit) atomicOr(&s_rowmask, rows_hit);
    }
   }
   __syncthreads();
  }
  if (s_wpop >= 0) flush(s_wpop, s_row0);
}

// FP32 push with four consecutive particles per thread: the state arrays are
// read and written as 128-bit vectors (five loads and five stores per four
// particles instead of twenty each), the chunk's first live row comes from
// loads already in flight, and absorbed or escaped particles are counted on a
// path taken only by warps that lost one.  Same chunks (2048 consecutive
// particles of one population, taken in groups from the counter), deposit
// window and per-particle arithmetic as k_push.  Population slot ranges start
// on multiples of four slots and extend to one (apic_create), so every vector
// lies inside its population's range; slots beyond the population's count
// are read and written back unchanged.
struct P4 {
  float4 x1, x2, vR, vZ, vT;
};

__device__ __forceinline__ float& lane4(float4& v, int k) { return k == 0 ? v.x : (k == 1 ? v.y : (k == 2 ? v.z : v.w)); }

template <bool kChord>
__global__ void __launch_bounds__(256, APIC_PUSH4_MIN_BLOCKS) k_push4(DevPtrs d, int win_n2, int win_rows, int group,
                                                                      int chunk_items) {
  extern __shared__ unsigned long long s_win[];
  const int win_words = 2 * win_rows * win_n2;
  const int plane = win_rows * win_n2;  // words of one plane of the window
  long long* s_pre = (long long*)(s_win + win_words);
  PushConst* s_pc = (PushConst*)(s_pre + d.n_pop + 1);
  __shared__ int s_row0, s_wpop, s_nsince, s_newrow0, s_flush, s_gi;
  __shared__ unsigned s_rowmask;
  constexpr int kPer = 4;                 // particles per thread and item
  const long long CH = (long long)chunk_items * blockDim.x;  // particles per chunk
  const int items = chunk_items / kPer;     // items of kPer x blockDim particles
  const int flush_chunks = (int)(65535 / CH);  // chunks between window flushes at most
  if (threadIdx.x == 0) {
    long long a = 0;
    for (int p = 0; p < d.n_pop; ++p) {
      s_pre[p] = a;
      a += (d.ps[p].n + CH - 1) / CH;
    }
    s_pre[d.n_pop] = a;
  }
  for (int p = threadIdx.x; p < d.n_pop; p += blockDim.x) {
    const Pop& P = d.pop[p];
    const Inst& I = d.inst[P.inst];
    PushConst C;
    C.al = (Real)I.alpha;
    C.h1 = (Real)I.h1;
    C.h2 = (Real)I.h2;
    C.x1_out = (Real)I.x1_out;
    C.dt = (Real)I.dt;
    C.B = (Real)I.B;
    C.h = Real(0.5) * (Real)(P.q / P.m) * (Real)I.dt;
    C.ih1 = (Real)(1.0 / I.h1);
    C.ih2 = (Real)(1.0 / I.h2);
    C.tz = C.h * (-(Real)I.B);
    C.sz = Real(2) * C.tz / (Real(1) + C.tz * C.tz);
    C.n1 = I.n1;
    C.n2 = I.n2;
    C.N2 = I.N2;
    C.fbits = P.fbits;
    C.node_off = I.node_off;
    C.acc_off = P.acc_off;
    s_pc[p] = C;
  }
  for (int k = threadIdx.x; k < win_words; k += blockDim.x) s_win[k] = 0ull;
  __syncthreads();
  const long long total_chunks = s_pre[d.n_pop];
  float4* X1 = (float4*)d.x1;
  float4* X2 = (float4*)d.x2;
  float4* VR = (float4*)d.vR;
  float4* VZ = (float4*)d.vZ;
  float4* VT = (float4*)d.vT;
  const float4* H = (const float4*)d.H;
  auto flush = [&](int wp, int row0) {
    const PushConst& Cw = s_pc[wp];
    const int rows = Cw.n2 <= win_n2 ? win_rows : 0;
    unsigned long long* g = d.acc + Cw.acc_off;
    const unsigned S = 1u << (Cw.fbits >> 1);
    const unsigned cm = s_rowmask;
    const unsigned nm = cm | (cm << 1);
    const int nrows = __popc(nm);
    for (int e = threadIdx.x; e < nrows * Cw.N2; e += blockDim.x) {
      const int q = e / Cw.N2, nj = e - q * Cw.N2;
      unsigned mm = nm;
      for (int z = 0; z < q; ++z) mm &= mm - 1u;
      const int rr = __ffs(mm) - 1;
      unsigned long long v = 0, w[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int cr = rr - (t & 1), cj = nj - (t >> 1);
        if (cr < 0 || cr >= rows || !((cm >> cr) & 1u) || cj < 0 || cj >= Cw.n2) continue;
        const unsigned long long* c = s_win + win_a(cr, cj, Cw.n2);
        if (c[win_m(plane)] == 0ull) continue;
        corner_weights(c[0], c[win_m(plane)], S, w);
        v += w[t];
      }
      if (v) atomicAdd(g + (long long)(row0 + rr) * Cw.N2 + nj, v);
    }
    __syncthreads();
    const int crows = __popc(cm);
    for (int e = threadIdx.x; e < 2 * crows * Cw.n2; e += blockDim.x) {
      const int q = e / (2 * Cw.n2), o = e - q * 2 * Cw.n2;
      unsigned mm = cm;
      for (int z = 0; z < q; ++z) mm &= mm - 1u;
      const int rz = __ffs(mm) - 1;
      s_win[o < Cw.n2 ? win_a(rz, o, Cw.n2) : win_a(rz, o - Cw.n2, Cw.n2) + win_m(plane)] = 0ull;
    }
    __syncthreads();
  };
  const int nch = (int)total_chunks;
  const int GS = group > 0 ? group : 1;
  const int ngroups = (nch + GS - 1) / GS;
  if (threadIdx.x == 0) {
    s_wpop = -1;
    s_nsince = 0;
    s_rowmask = 0u;
  }
  __syncthreads();
  const unsigned lane = threadIdx.x & 31;
  for (int q = 0;; ++q) {
    if (q % GS == 0) {
      __syncthreads();  // every warp has read the previous group's index
      if (threadIdx.x == 0) s_gi = (int)atomicAdd((unsigned long long*)(d.cnt + 1), 1ull);
      __syncthreads();
    }
    const int gi = s_gi;
    if (gi >= ngroups) break;
    const long long chunk = (long long)gi * GS + q % GS;
    if (chunk >= nch) continue;
    const int pop = find_pop(s_pre, d.n_pop, chunk);
    const PushConst C = s_pc[pop];
    const long long npop = d.ps[pop].n, pbase = d.pop[pop].base;
    const long long c0 = (chunk - s_pre[pop]) * CH;
    const long long v0 = (pbase + c0) / kPer + threadIdx.x;  // vector of item 0 (pbase, c0: multiples of 4)
    const int nleft = npop - c0 > CH ? (int)CH : (int)(npop - c0);  // particles of the chunk in the population
    P4 st;
    auto load = [&](int it) {
      const long long v = v0 + (long long)it * blockDim.x;
      if ((it * (int)blockDim.x + (int)threadIdx.x) * kPer < nleft) {
        st.x1 = X1[v];
        st.x2 = X2[v];
        st.vR = VR[v];
        st.vZ = VZ[v];
        st.vT = VT[v];
      } else {
        st.x1 = make_float4(2.0f, 2.0f, 2.0f, 2.0f);
      }
    };
    load(0);
    if (threadIdx.x == 0) {
      // window rows from the chunk's first live particle (this thread holds the first four)
      int row = -1;
      // (the window's place changes no result: deposits outside it go to
      // the global accumulator)
      for (int k = 0; k < kPer && row < 0; ++k) {
        const float xq = lane4(st.x1, k);
        if (k < nleft && xq < 0.0f) row = (int)floorf((xq + 1.0f) * C.ih1);
      }
      for (int qq = kPer; row < 0 && qq < 64 && c0 + qq < npop; ++qq) {
        const float xq = ((const float*)d.x1)[pbase + c0 + qq];
        if (xq < 0.0f) row = (int)floorf((xq + 1.0f) * C.ih1);
      }
      row = row < 0 ? 0 : row;
      const int r0 = row > 0 ? row - 1 : 0;
      const int rows = C.n2 <= win_n2 ? win_rows : 0;
      const bool keep = s_wpop == pop && s_nsince < flush_chunks && r0 >= s_row0 && r0 + 2 < s_row0 + rows;
      s_flush = s_wpop >= 0 && !keep;
      s_newrow0 = keep ? s_row0 : r0;
    }
    __syncthreads();
    if (s_flush) flush(s_wpop, s_row0);
    if (threadIdx.x == 0) {
      if (s_row0 != s_newrow0 || s_wpop != pop || s_flush) {
        s_row0 = s_newrow0;
        s_wpop = pop;
        s_rowmask = 0u;
        s_nsince = 0;
      }
      s_nsince += 1;
    }
    __syncthreads();
    CellWin CW;
    CW.s = s_win;
    CW.plane = plane;
    CW.g = d.acc + C.acc_off;
    CW.row0 = s_row0;
    CW.rows = C.n2 <= win_n2 ? win_rows : 0;
    CW.n2 = C.n2;
    CW.N2 = C.N2;
    const float4* Hi = H + C.node_off;
    const int bits = C.fbits >> 1;
    for (int it = 0; it < items; ++it) {
      if (it > 0) load(it);
      const int base_local = it * (int)blockDim.x * kPer + (int)threadIdx.x * kPer;  // chunk-local index of particle 0
      unsigned deadm = 0u, absm = 0u, rows_hit = 0u;
#pragma unroll
      for (int k = 0; k < kPer; ++k) {
        const bool active = base_local + k < nleft;
        const float x1 = lane4(st.x1, k);
        const bool alive = active && x1 < 0.0f;
        int fate = 0;
        int key = -1, di = 0, dj = 0;
        unsigned q1 = 0, q2 = 0;
        if (alive) {
          float x2 = lane4(st.x2, k), vR = lane4(st.vR, k), vZ = lane4(st.vZ, k), vT = lane4(st.vT, k);
          const float al = C.al, dt = C.dt;
          float x1f = x1;
          float disc = 1.0f - 4.0f * al * x1f * x2;
          float ir = __fdividef(-2.0f * x1f, 1.0f + sqrtf(disc));  // 1/r (Eq. 3)
          float r = __fdividef(1.0f, ir);
          float s2 = (1.0f - x2) * (1.0f + x2);
          float sn = sqrtf(s2);
          float R = r * sn, Z = r * x2;
          float u1 = (x1f + 1.0f) * C.ih1, u2 = (x2 + 1.0f) * C.ih2;
          int ci = min(max((int)floorf(u1), 0), C.n1 - 1), cj = min(max((int)floorf(u2), 0), C.n2 - 1);
          float f1 = fminf(fmaxf(u1 - (float)ci, 0.0f), 1.0f), f2 = fminf(fmaxf(u2 - (float)cj, 0.0f), 1.0f);
          const int n00 = ci * C.N2 + cj;
          const float4 b0 = Hi[n00], b1 = Hi[n00 + C.N2];  // (G00, G01), (G10, G11)
          float g1 = (1.0f - f2) * ((1.0f - f1) * b0.x + f1 * b1.x) + f2 * ((1.0f - f1) * b0.z + f1 * b1.z);
          float g2 = (1.0f - f2) * ((1.0f - f1) * b0.y + f1 * b1.y) + f2 * ((1.0f - f1) * b0.w + f1 * b1.w);
          float ir3 = ir * ir * ir;
          float x1R = sn * (r + 3.0f * al * x2) * ir3, x1Z = (r * x2 + al * (3.0f * x2 * x2 - 1.0f)) * ir3;
          float x2R = -x2 * sn * ir, x2Z = s2 * ir;
          float ER = -(x1R * g1 + x2R * g2), EZ = -(x1Z * g1 + x2Z * g2);
          float h = C.h, tz = C.tz, sz = C.sz;
          float vx = vR + h * ER, vy = vT, vz = vZ + h * EZ;
          float px_ = vx + vy * tz, py_ = vy - vx * tz;
          vx = vx + py_ * sz + h * ER;
          vy = vy - px_ * sz;
          vz = vz + h * EZ;
          float Xc = R + vx * dt, Yc = vy * dt, Zn = Z + vz * dt;
          float Rn2 = Xc * Xc + Yc * Yc;
          float cr = 1.0f, sr = 0.0f;
          if (Rn2 > 0.0f) {
            float iR = rsqrtf(Rn2);
            cr = Xc * iR;
            sr = Yc * iR;
          }
          float vRn = cr * vx + sr * vy, vTn = -sr * vx + cr * vy;
          float rn2 = Rn2 + Zn * Zn;
          float irn = rsqrtf(rn2);
          float rn = rn2 * irn;
          float x2n = Zn * irn;
          float tr = 2.0f * rn - 1.0f;
          bool hit = tr < 0.0f || tr * tr < 1.0f + 4.0f * al * x2n;
          float tau = dt;
          if (kChord && !hit && (d.inst[d.pop[pop].inst].flags & APIC_CHORD_ABSORB)) {
            const float se = chord_entry(al, R, Z, vx * dt, vy * dt, vz * dt);
            if (se > 0.0f) {
              hit = true;
              tau = dt * se;
            }
          }
          if (hit) {
            const Pop& P = d.pop[pop];
            absorb_tally(d, d.inst[P.inst], P, R, Z, vx, vz, vy, tau);
            lane4(st.x1, k) = 2.0f;
            fate = 1;
          } else {
            float x1n = -irn * (1.0f + al * x2n * irn);
            if (x1n > C.x1_out) {
              lane4(st.x1, k) = 2.0f;
              fate = 2;
            } else {
              lane4(st.x1, k) = x1n;
              lane4(st.x2, k) = x2n;
              lane4(st.vR, k) = vRn;
              lane4(st.vZ, k) = vz;
              lane4(st.vT, k) = vTn;
              float v1 = (x1n + 1.0f) * C.ih1, v2 = (x2n + 1.0f) * C.ih2;
              int ni = min(max((int)floorf(v1), 0), C.n1 - 1), nj = min(max((int)floorf(v2), 0), C.n2 - 1);
              float e1 = fminf(fmaxf(v1 - (float)ni, 0.0f), 1.0f), e2 = fminf(fmaxf(v2 - (float)nj, 0.0f), 1.0f);
              const float one = (float)(1u << bits);
              q1 = min((unsigned)(e1 * one + 0.5f), 1u << bits);
              q2 = min((unsigned)(e2 * one + 0.5f), 1u << bits);
              key = ni * C.N2 + nj;
              di = ni;
              dj = nj;
            }
          }
        }
        if (fate) {
          deadm |= 1u << k;
          if (fate == 1) absm |= 1u << k;
        }
        deposit_moments(CW, key, di, dj, q1, q2, bits, key >= 0);
        const int rr = di - CW.row0;
        if (key >= 0 && rr >= 0 && rr < CW.rows) rows_hit |= 1u << rr;
      }
      if ((it * (int)blockDim.x + (int)threadIdx.x) * kPer < nleft) {
        const long long v = v0 + (long long)it * blockDim.x;
        X1[v] = st.x1;
        X2[v] = st.x2;
        VR[v] = st.vR;
        VZ[v] = st.vZ;
        VT[v] = st.vT;
      }
      const unsigned rh = __reduce_or_sync(kFull, rows_hit);
      if (lane == 0 && rh) atomicOr(&s_rowmask, rh);
      // absorbed or escaped particles: counters and freed slots (rare)
      if (__any_sync(kFull, deadm != 0u)) {
        const unsigned nd = __popc(deadm);
        unsigned incl = nd;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const unsigned y = __shfl_up_sync(kFull, incl, o);
          if ((int)lane >= o) incl += y;
        }
        const unsigned tot = __shfl_sync(kFull, incl, 31);
        const unsigned tabs = __reduce_add_sync(kFull, __popc(absm));
        long long h0 = 0;
        if (lane == 0) {
          PopState& S = d.ps[pop];
          if (tabs) atomicAdd((unsigned long long*)&S.absorbed, (unsigned long long)tabs);
          if (tot - tabs) atomicAdd((unsigned long long*)&S.escaped, (unsigned long long)(tot - tabs));
          h0 = (long long)atomicAdd((unsigned long long*)&S.n_holes, (unsigned long long)tot);
        }
        h0 = __shfl_sync(kFull, h0, 0);
        long long hpos = h0 + (long long)(incl - nd);
        for (int k = 0; k < kPer; ++k)
          if ((deadm >> k) & 1u) d.holes[d.pop[pop].base + hpos++] = (int32_t)(c0 + base_local + k);
      }
    }
    __syncthreads();
  }
  if (s_wpop >= 0) flush(s_wpop, s_row0);
}

// Deposit every live particle (after external changes to the particle set,
// and in every step of the sensitivity window).  Each CTA takes a contiguous
// range of the (row-sorted) particles in chunks of kDepItems x blockDim and
// adds the corner weights into a shared-memory window of kWinRows node rows
// of one population, flushed to the global accumulator only when a chunk's
// first row or population leaves it; corners outside the window go to global
// memory directly.  Integer sums: the result does not depend on the order.
constexpr int kDepItems = 8;
__global__ void __launch_bounds__(256) k_deposit_all(DevPtrs d, int win_n2) {
  extern __shared__ unsigned long long s_dw[];  // [kWinRows][win_n2 + 1]
  __shared__ long long s_pre[kMaxPop + 1];
  __shared__ int s_row0, s_wpop, s_newrow0, s_newpop, s_flush;
  if (threadIdx.x == 0) {
    long long a = 0;
    for (int p = 0; p < d.n_pop; ++p) {
      s_pre[p] = a;
      a += d.ps[p].n;
    }
    s_pre[d.n_pop] = a;
    s_wpop = -1;
  }
  const int WN = win_n2 + 1;
  for (int k = threadIdx.x; k < kWinRows * WN; k += blockDim.x) s_dw[k] = 0ull;
  __syncthreads();
  const long long total = s_pre[d.n_pop];
  const Real* X1 = (const Real*)d.x1;
  const Real* X2 = (const Real*)d.x2;
  const long long CH = (long long)kDepItems * blockDim.x;
  const long long nch = (total + CH - 1) / CH;
  const long long per = (nch + gridDim.x - 1) / gridDim.x;
  const long long cb = (long long)blockIdx.x * per, ce = cb + per < nch ? cb + per : nch;
  auto flush = [&](int wp, int row0) {
    const Pop& P = d.pop[wp];
    const Inst& I = d.inst[P.inst];
    const int rows = I.n2 <= win_n2 ? kWinRows : 0;
    unsigned long long* g = d.acc + P.acc_off;
    for (int e = threadIdx.x; e < rows * I.N2; e += blockDim.x) {
      const int r = e / I.N2, j = e - r * I.N2;
      const unsigned long long v = s_dw[r * WN + j];
      if (v && row0 + r <= I.n1) {
        atomicAdd(g + (long long)(row0 + r) * I.N2 + j, v);
        s_dw[r * WN + j] = 0ull;
      }
    }
    __syncthreads();
  };
  for (long long ch = cb; ch < ce; ++ch) {
    const long long t0 = ch * CH;
    if (threadIdx.x == 0) {
      // window rows from the chunk's first live particle
      int pop = find_pop(s_pre, d.n_pop, t0), row = 0;
      for (long long q = t0; q < t0 + 64 && q < total; ++q) {
        const int pq = find_pop(s_pre, d.n_pop, q);
        const Real xq = X1[d.pop[pq].base + (q - s_pre[pq])];
        if (xq < Real(0)) {
          pop = pq;
          row = (int)floor((double)((xq + Real(1)) / (Real)d.inst[d.pop[pq].inst].h1));
          break;
        }
      }
      const int r0 = row > 0 ? row - 1 : 0;
      const bool keep = s_wpop == pop && r0 >= s_row0 && r0 + 2 < s_row0 + kWinRows;
      s_flush = s_wpop >= 0 && !keep;
      s_newrow0 = keep ? s_row0 : r0;
      s_newpop = pop;
    }
    __syncthreads();
    if (s_flush) flush(s_wpop, s_row0);
    if (threadIdx.x == 0) {
      s_row0 = s_newrow0;
      s_wpop = s_newpop;
    }
    __syncthreads();
    const int wpop = s_wpop, row0 = s_row0;
    for (int it = 0; it < kDepItems; ++it) {
      const long long t = t0 + (long long)it * blockDim.x + threadIdx.x;
      if (t >= total) break;
      const int pop = find_pop(s_pre, d.n_pop, t);
      const Pop& P = d.pop[pop];
      const Inst& I = d.inst[P.inst];
      const long long slot = P.base + (t - s_pre[pop]);
      const Real x1 = X1[slot];
      if (!(x1 < Real(0))) continue;
      const Cell c = locate(I, x1, X2[slot]);
      const W4 w = weights(c, P.fbits);
      const int rr = c.i - row0;
      if (pop == wpop && I.n2 <= win_n2 && rr >= 0 && rr + 1 < kWinRows) {
        unsigned long long* sw = s_dw + rr * WN + c.j;
        if (w.w00) atomicAdd(sw, w.w00);
        if (w.w10) atomicAdd(sw + WN, w.w10);
        if (w.w01) atomicAdd(sw + 1, w.w01);
        if (w.w11) atomicAdd(sw + WN + 1, w.w11);
      } else {
        unsigned long long* g = d.acc + dep_key(I, P, c);
        if (w.w00) atomicAdd(g, w.w00);
        if (w.w10) atomicAdd(g + I.N2, w.w10);
        if (w.w01) atomicAdd(g + 1, w.w01);
        if (w.w11) atomicAdd(g + I.N2 + 1, w.w11);
      }
    }
    __syncthreads();
  }
  if (s_wpop >= 0) flush(s_wpop, s_row0);
}

// Initial load, uniform in physical volume: x2 from the inverse CDF of
// (r_out^3 - r_g^3)(x2) (Eq. 5 integrated along x1), r by inverting the r^3
// cumulative, velocity Maxwellian at T (three Box-Muller normals).
__global__ void k_load(DevPtrs d, int pop, long long n0, long long count, long long draw0) {
  long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= count) return;
  const Pop& P = d.pop[pop];
  const Inst& I = d.inst[P.inst];
  uint32_t u[8];
  draws8(I, P, draw0 + k, 1u, u);
  Real al = (Real)I.alpha;
  Real x2 = sample_x2(d.tab + I.tab_off, d.guide + I.tab_off, unit(u[0]));
  Real rg = r_grain(al, x2), ro = radius(al, (Real)I.x1_out, x2);
  Real r3 = rg * rg * rg + unit(u[1]) * (ro * ro * ro - rg * rg * rg);
  Real r = cbrt(r3);
  Real ra = sqrt(Real(-2) * log(unit(u[2]))), rb = sqrt(Real(-2) * log(unit(u[4])));
  Real pa = Real(2 * kPi) * unit(u[3]), pb = Real(2 * kPi) * unit(u[5]);
  Real vth = (Real)P.vth;
  long long slot = P.base + n0 + k;
  ((Real*)d.x1)[slot] = x1_at(al, r, x2);
  ((Real*)d.x2)[slot] = x2;
  ((Real*)d.vR)[slot] = vth * (ra * cos(pa));
  ((Real*)d.vZ)[slot] = vth * (ra * sin(pa));
  ((Real*)d.vT)[slot] = vth * (rb * cos(pb));
}

__global__ void k_explicit(DevPtrs d, int pop, long long n0, long long count, const double* st) {
  long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= count) return;
  long long slot = d.pop[pop].base + n0 + k;
  ((Real*)d.x1)[slot] = (Real)st[5 * k + 0];
  ((Real*)d.x2)[slot] = (Real)st[5 * k + 1];
  ((Real*)d.vR)[slot] = (Real)st[5 * k + 2];
  ((Real*)d.vZ)[slot] = (Real)st[5 * k + 3];
  ((Real*)d.vT)[slot] = (Real)st[5 * k + 4];
}

// Surface injection (Sec. 1, Eq. 4): x2 from the inverse CDF of dA/dx2 on
// x1 = x1_out, flux-weighted half-Maxwellian along the inward normal
// -grad x1 / |grad x1|, Maxwellian along the meridional tangent and Theta,
// free flight for a uniform fraction of dt, then absorption / escape tests.
// Stored particles fill freed slots first, then extend the population.
__global__ void __launch_bounds__(256) k_inject(DevPtrs d) {
  // The injected particles land within a cell row or two of the outer
  // surface: their corner weights are summed in a shared-memory window of the
  // last kInjRows node rows and added to the global accumulator once per CTA
  // (every particle's weights on the same few hundred nodes would otherwise
  // serialise on them).
  __shared__ unsigned long long s_nodes[kInjRows * (kInjMaxN2 + 1)];
  const int pop = blockIdx.y;
  PopState& S = d.ps[pop];
  const Pop& P = d.pop[pop];
  const Inst& I = d.inst[P.inst];
  const long long n_inj = S.n_inj;
  const int wrow0 = I.n1 + 1 - kInjRows;  // first node row of the window
  const bool win = I.N2 <= kInjMaxN2 + 1;
  for (int e = threadIdx.x; e < kInjRows * I.N2 && win; e += blockDim.x) s_nodes[e] = 0ull;
  __syncthreads();
  for (long long base = (long long)blockIdx.x * blockDim.x; base < n_inj; base += (long long)gridDim.x * blockDim.x) {
  const long long k = base + threadIdx.x;
  bool active = k < n_inj;
  long long key = -1;
  W4 w = {0, 0, 0, 0};
  int ci = 0, cj = 0;
  int fate = 0;  // 1 absorbed, 2 escaped, 3 stored
  Real x1n = Real(0), x2n = Real(0), vRn = Real(0), vZn = Real(0), vTn = Real(0);
  if (active) {
    uint32_t u[8];
    draws8(I, P, S.draws + k, 2u, u);
    Real al = (Real)I.alpha, dt = (Real)I.dt;
    Real x2 = sample_x2(d.tab + I.tab_off + (kTable + 1), d.guide + I.tab_off + (kTable + 1), unit(u[0]));
    Real vth = (Real)P.vth;
    Real vn = vth * sqrt(Real(-2) * log(unit(u[1])));
    Real ra = sqrt(Real(-2) * log(unit(u[2])));
    Real pa = Real(2 * kPi) * unit(u[3]);
    Real vt = vth * (ra * cos(pa)), vth_ = vth * (ra * sin(pa));
    Real tau = unit(u[4]) * dt;
    Real r = radius(al, (Real)I.x1_out, x2);
    Real sn = sqrt((Real(1) - x2) * (Real(1) + x2));
    Real R = r * sn, Z = r * x2;
    Metric<Real> m = metric(al, r, x2);
    Real gn = sqrt(m.x1R * m.x1R + m.x1Z * m.x1Z);
    Real nR = -m.x1R / gn, nZ = -m.x1Z / gn;
    Real tR = nZ, tZ = -nR;
    Real vx = vn * nR + vt * tR, vz = vn * nZ + vt * tZ, vy = vth_;
    Real Xc = R + vx * tau, Yc = vy * tau, Zn = Z + vz * tau;
    Real Rn = sqrt(Xc * Xc + Yc * Yc);
    Real cr = Real(1), sr = Real(0);
    if (Rn > Real(0)) {
      cr = Xc / Rn;
      sr = Yc / Rn;
    }
    Real rn = sqrt(Rn * Rn + Zn * Zn);
    x2n = Zn / rn;
    bool hit = rn < r_grain(al, x2n);
    Real tau_in = tau;  // flight time up to a point inside the grain
    if (!hit && (I.flags & APIC_CHORD_ABSORB)) {
      const Real se = chord_entry(al, R, Z, vx * tau, vy * tau, vz * tau);
      if (se > Real(0)) {
        hit = true;
        tau_in = tau * se;
      }
    }
    if (hit) {
      absorb_tally(d, I, P, R, Z, vx, vz, vy, tau_in);
      fate = 1;
    } else {
      x1n = x1_at(al, rn, x2n);
      if (x1n > (Real)I.x1_out) {
        fate = 2;
      } else {
        fate = 3;
        vRn = cr * vx + sr * vy;
        vZn = vz;
        vTn = -sr * vx + cr * vy;
      }
    }
  }
  // warp-aggregated counters: one atomic per warp and outcome (the storage
  // counter is shared by every injected particle of the population)
  const unsigned lane = threadIdx.x & 31, lt = (1u << lane) - 1u;
  const unsigned m_abs = __ballot_sync(kFull, fate == 1), m_esc = __ballot_sync(kFull, fate == 2);
  const unsigned m_st = __ballot_sync(kFull, fate == 3);
  if (lane == 0) {
    if (m_abs) atomicAdd((unsigned long long*)&S.absorbed, (unsigned long long)__popc(m_abs));
    if (m_esc) atomicAdd((unsigned long long*)&S.escaped, (unsigned long long)__popc(m_esc));
  }
  long long sbase = 0;
  if (m_st) {
    const int leader = __ffs(m_st) - 1;
    if ((int)lane == leader) sbase = (long long)atomicAdd((unsigned long long*)&S.inj_stored, (unsigned long long)__popc(m_st));
    sbase = __shfl_sync(kFull, sbase, leader);
  }
  if (fate == 3) {
    const long long sidx = sbase + __popc(m_st & lt);
    const long long nh = S.n_holes, n = S.n;
    const long long kk = sidx < nh ? d.holes[P.base + nh - 1 - sidx] : n + (sidx - nh);
    if (kk >= P.cap) {
      atomicAdd((unsigned long long*)&S.dropped, 1ull);
      atomicOr(d.err, kErrCapacity);
    } else {
      long long slot = P.base + kk;
      ((Real*)d.x1)[slot] = x1n;
      ((Real*)d.x2)[slot] = x2n;
      ((Real*)d.vR)[slot] = vRn;
      ((Real*)d.vZ)[slot] = vZn;
      ((Real*)d.vT)[slot] = vTn;
      Cell c = locate(I, x1n, x2n);
      key = dep_key(I, P, c);
      ci = c.i;
      cj = c.j;
      w = weights(c, P.fbits);
    }
  }
  if (key >= 0) {
    if (win && ci >= wrow0) {
      unsigned long long* sn0 = s_nodes + (ci - wrow0) * I.N2 + cj;
      if (w.w00) atomicAdd(sn0, w.w00);
      if (w.w10) atomicAdd(sn0 + I.N2, w.w10);
      if (w.w01) atomicAdd(sn0 + 1, w.w01);
      if (w.w11) atomicAdd(sn0 + I.N2 + 1, w.w11);
    } else {
      if (w.w00) atomicAdd(d.acc + key, w.w00);
      if (w.w10) atomicAdd(d.acc + key + I.N2, w.w10);
      if (w.w01) atomicAdd(d.acc + key + 1, w.w01);
      if (w.w11) atomicAdd(d.acc + key + I.N2 + 1, w.w11);
    }
  }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < kInjRows * I.N2 && win; e += blockDim.x) {
    const unsigned long long v = s_nodes[e];
    if (v) atomicAdd(d.acc + P.acc_off + (long long)wrow0 * I.N2 + e, v);
  }
}

// ---------------------------------------------------------------------------
// Counting sort of every population by grid row (the push's deposit window
// covers whole rows), which also drops freed slots: count -> exclusive scan
// over all (population, row) bins -> scatter into the second buffer.  The
// count reads x1 alone as 16-byte vectors and counts runs of equal rows in
// registers; the scatter streams its chunks' states through shared memory
// with bulk asynchronous copies issued a chunk ahead.  Both touch the global
// counters once per row a CTA's share or chunk holds (recently sorted
// particles: one to three rows).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void chunk_prefix(const DevPtrs& d, long long CH, long long* pre) {
  if (threadIdx.x == 0) {
    long long a = 0;
    for (int p = 0; p < d.n_pop; ++p) {
      pre[p] = a;
      a += (d.ps[p].n + CH - 1) / CH;
    }
    pre[d.n_pop] = a;
  }
  __syncthreads();
}

// Warp-aggregated shared-memory increment of counter[key] by one per lane;
// returns the lane's rank among the lanes of its key (keys < 0: no-op).
__device__ __forceinline__ unsigned warp_count(unsigned* counter, int key) {
  const int lane = threadIdx.x & 31;
  unsigned grp = __match_any_sync(kFull, key);
  int leader = __ffs(grp) - 1;
  unsigned rank = __popc(grp & ((1u << lane) - 1u));
  unsigned base = 0;
  if (key >= 0 && lane == leader) base = atomicAdd(counter + key, (unsigned)__popc(grp));
  base = __shfl_sync(kFull, base, leader);
  return base + rank;
}

// Exclusive scan of cell_cnt into cell_off: per-block scan (1024 cells) ...
__global__ void __launch_bounds__(1024) k_scan_blocks(DevPtrs d) {
  __shared__ unsigned long long ws[32];
  long long c = (long long)blockIdx.x * 1024 + threadIdx.x;
  unsigned long long v = c < d.total_cells ? d.cell_cnt[c] : 0ull;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned long long x = v;
  for (int o = 1; o < 32; o <<= 1) {
    unsigned long long up = __shfl_up_sync(kFull, x, o);
    if (lane >= o) x += up;
  }
  if (lane == 31) ws[warp] = x;
  __syncthreads();
  if (warp == 0) {
    unsigned long long y = ws[lane];
    for (int o = 1; o < 32; o <<= 1) {
      unsigned long long up = __shfl_up_sync(kFull, y, o);
      if (lane >= o) y += up;
    }
    ws[lane] = y;
  }
  __syncthreads();
  unsigned long long excl = x - v + (warp > 0 ? ws[warp - 1] : 0ull);
  if (c < d.total_cells) d.cell_off[c] = excl;
  if (threadIdx.x == 1023) d.scan_tmp[blockIdx.x] = excl + v;
}

// ... scan of the block sums (one CTA) ...
__global__ void __launch_bounds__(1024) k_scan_top(DevPtrs d, int nblocks) {
  __shared__ unsigned long long sh[1024];
  // sequential carry over chunks of 1024 block sums
  unsigned long long carry = 0;
  for (int c0 = 0; c0 < nblocks; c0 += 1024) {
    int k = c0 + threadIdx.x;
    unsigned long long v = k < nblocks ? d.scan_tmp[k] : 0ull;
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
      unsigned long long add = threadIdx.x >= o ? sh[threadIdx.x - o] : 0ull;
      __syncthreads();
      sh[threadIdx.x] += add;
      __syncthreads();
    }
    if (k < nblocks) d.scan_tmp[k] = carry + sh[threadIdx.x] - v;  // exclusive
    unsigned long long tot = sh[1023];
    __syncthreads();
    carry += tot;
  }
  if (threadIdx.x == 0) d.cell_off[d.total_cells] = carry;
}

// ... and the block offsets added back; the counters are cleared for the scatter.
__global__ void __launch_bounds__(1024) k_scan_add(DevPtrs d) {
  long long c = (long long)blockIdx.x * 1024 + threadIdx.x;
  if (c < d.total_cells) {
    d.cell_off[c] += d.scan_tmp[blockIdx.x];
    d.cell_cnt[c] = 0u;
  }
}

// Grid row of a stored x1 (row -1: a freed slot, x1 > 0), one expression for
// the count and the scatter so that both place every particle in the same row.
__device__ __forceinline__ int sort_row(Real x, Real ih1, int nrows) {
  if (!(x < Real(0))) return -1;
  int row = (int)floor((x + Real(1)) * ih1);
  return row < 0 ? 0 : (row > nrows - 1 ? nrows - 1 : row);
}

// A population's constants of the sort, read once per CTA.
struct SortConst {
  long long base, cell_off, n;
  Real ih1;  // 1 / h1 in the particle precision (the row key only orders the particles)
  int nrows;
};

__device__ __forceinline__ void sort_consts(const DevPtrs& d, SortConst* sc) {
  for (int p = threadIdx.x; p < d.n_pop; p += blockDim.x) {
    const Pop& P = d.pop[p];
    const Inst& I = d.inst[P.inst];
    sc[p] = SortConst{P.base, P.cell_off, d.ps[p].n, (Real)(1.0 / I.h1), I.n1};
  }
}

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;

// 16-byte vectors of the particle precision (a population's slot range
// starts on a 16-byte boundary and holds a multiple of four slots).
template <class T>
struct Vec16;
template <>
struct Vec16<float> {
  using T = float4;
  static constexpr int kN = 4;
  __device__ static float get(const float4& v, int k) { return k == 0 ? v.x : k == 1 ? v.y : k == 2 ? v.z : v.w; }
};
template <>
struct Vec16<double> {
  using T = double2;
  static constexpr int kN = 2;
  __device__ static double get(const double2& v, int k) { return k == 0 ? v.x : v.y; }
};
using RealV = Vec16<Real>;

// Count pass: every CTA takes a contiguous share of the populations' slots
// laid end to end (whole 16-byte vectors, kCountUnroll of them in flight per
// thread; a share spans one or a few populations), counts runs of equal rows
// in registers (recently sorted particles change row rarely), adds a run to a
// shared-memory histogram when it ends, and adds the histogram's rows
// [lo, hi] to cell_cnt once per population of the share.
constexpr int kCountUnroll = 4;

__global__ void __launch_bounds__(kSortThreads) k_sort_count(DevPtrs d, int hist_rows) {
  extern __shared__ unsigned hist[];  // [hist_rows]
  __shared__ SortConst sc[kMaxPop];
  __shared__ int s_lo[2], s_hi[2];  // population p's row range in [p & 1] (reset for p + 2)
  __shared__ long long gpre[kMaxPop + 1];  // vectors of the populations before p
  sort_consts(d, sc);
  for (int r = threadIdx.x; r < hist_rows; r += blockDim.x) hist[r] = 0u;
  if (threadIdx.x < 2) {
    s_lo[threadIdx.x] = INT_MAX;
    s_hi[threadIdx.x] = -1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    long long a = 0;
    for (int p = 0; p < d.n_pop; ++p) {
      gpre[p] = a;
      a += (sc[p].n + RealV::kN - 1) / RealV::kN;
    }
    gpre[d.n_pop] = a;
  }
  __syncthreads();
  const long long total = gpre[d.n_pop];
  const long long per = (total + gridDim.x - 1) / gridDim.x;
  const long long G0 = (long long)blockIdx.x * per, G1 = min(total, G0 + per);
  if (G0 >= G1) return;  // (uniform over the CTA)
  const int p0 = find_pop(gpre, d.n_pop, G0), p1 = find_pop(gpre, d.n_pop, G1 - 1);
  for (int pop = p0; pop <= p1; ++pop) {
    const SortConst P = sc[pop];
    const typename RealV::T* X = (const typename RealV::T*)((const Real*)d.x1 + P.base);
    const long long g0 = max(G0, gpre[pop]) - gpre[pop], g1 = min(G1, gpre[pop + 1]) - gpre[pop];
    int run = -1, len = 0, lo = INT_MAX, hi = -1;
    for (long long g = g0 + threadIdx.x; g < g1; g += (long long)kCountUnroll * kSortThreads) {
      typename RealV::T v[kCountUnroll];
#pragma unroll
      for (int u = 0; u < kCountUnroll; ++u) {
        const long long gu = g + (long long)u * kSortThreads;
        if (gu < g1) v[u] = X[gu];
      }
#pragma unroll
      for (int u = 0; u < kCountUnroll; ++u) {
        const long long gu = g + (long long)u * kSortThreads;
#pragma unroll
        for (int k = 0; k < RealV::kN; ++k) {
          const int row = gu < g1 && gu * RealV::kN + k < P.n ? sort_row(RealV::get(v[u], k), P.ih1, P.nrows) : -1;
          if (row >= 0) {
            if (row != run) {
              if (len) atomicAdd(hist + run, (unsigned)len);
              run = row;
              len = 0;
            }
            ++len;
            lo = min(lo, row);
            hi = max(hi, row);
          }
        }
      }
    }
    if (len) atomicAdd(hist + run, (unsigned)len);
    lo = __reduce_min_sync(kFull, lo);
    hi = __reduce_max_sync(kFull, hi);
    if ((threadIdx.x & 31) == 0 && hi >= 0) {
      atomicMin(&s_lo[pop & 1], lo);
      atomicMax(&s_hi[pop & 1], hi);
    }
    __syncthreads();
    // no live particle: the empty range [0, -1]
    const int r1 = s_hi[pop & 1], r0 = r1 >= 0 ? s_lo[pop & 1] : 0;
    for (int r = r0 + threadIdx.x; r <= r1; r += blockDim.x) {
      const unsigned c = hist[r];
      if (c) {
        atomicAdd(d.cell_cnt + P.cell_off + r, c);
        hist[r] = 0u;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      s_lo[pop & 1] = INT_MAX;
      s_hi[pop & 1] = -1;
    }
  }
}

// Scatter pass: chunks of kScatterItems x 256 consecutive slots of one
// population, the five state arrays of a CTA's next chunks streamed into
// shared-memory stages by bulk asynchronous copies while it places the
// current one.
constexpr int kScatterItems = 8;
constexpr int kScatterChunk = kScatterItems * kSortThreads;
constexpr int kScatterStages = 2;
constexpr int kScatterStageBytes = 5 * kScatterChunk * (int)sizeof(Real);
static_assert(kScatterItems * kSortWarps % 32 == 0, "whole entries per lane in the chunk-order prefix");

static int scatter_smem(int hist_rows) {
  return kScatterStages * kScatterStageBytes + 2 * hist_rows * (int)sizeof(unsigned);
}

// Bulk copies of chunk `chunk`'s state arrays into a stage (thread 0).  The
// population's slot range starts on a 16-byte boundary and holds a multiple
// of four slots, so the copy rounded up to whole 16-byte units stays inside it.
__device__ __forceinline__ void scatter_issue(const DevPtrs& d, const long long* pre, const SortConst* sc,
                                              long long chunk, Real* stage, uint64_t* bar) {
  const int pop = find_pop(pre, d.n_pop, chunk);
  const SortConst& P = sc[pop];
  const long long c0 = (chunk - pre[pop]) * kScatterChunk;
  const long long n = min((long long)kScatterChunk, P.n - c0);
  const unsigned bytes = (unsigned)(((n + 3) & ~3ll) * (long long)sizeof(Real));
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  mbar_expect_tx(bar, 5u * bytes);
  const Real* src[5] = {(const Real*)d.x1, (const Real*)d.x2, (const Real*)d.vR, (const Real*)d.vZ,
                        (const Real*)d.vT};
#pragma unroll
  for (int a = 0; a < 5; ++a) bulk_g2s(stage + a * kScatterChunk, src[a] + P.base + c0, bytes, bar);
}

// The chunks blockIdx.x, blockIdx.x + gridDim.x, ... of every population:
// each reserves its range of every row it holds (cell_off + an atomic on
// cell_cnt, which the scan cleared) and writes its live particles there in
// the second buffer.  Recently sorted particles put most chunks in one row:
// its range is the chunk's live particles and their positions follow the
// chunk order (ballots, then an exclusive prefix over the (item, warp)
// blocks); a chunk over several rows counts and places per row in shared
// memory.  A copy that never lands sets kErrTimeout, and the CTA leaves after
// the copies still in flight.
__global__ void __launch_bounds__(kSortThreads) k_sort_scatter(DevPtrs d, int hist_rows) {
  extern __shared__ __align__(128) unsigned char s_raw[];
  Real* stages = (Real*)s_raw;
  unsigned* cnt = (unsigned*)(s_raw + (size_t)kScatterStages * kScatterStageBytes);
  unsigned* cur = cnt + hist_rows;  // the chunk's next position in each row
  __shared__ long long pre[kMaxPop + 1];
  __shared__ SortConst sc[kMaxPop];
  __shared__ __align__(8) uint64_t bar[kScatterStages];
  __shared__ int s_r0, s_r1;        // rows of the chunk: [s_r0, s_r1]
  __shared__ unsigned s_base;       // first position of a one-row chunk
  __shared__ unsigned s_wc[kScatterItems * kSortWarps];  // live particles per (item, warp), then their prefix
  sort_consts(d, sc);
  chunk_prefix(d, kScatterChunk, pre);  // (its barrier publishes sc too)
  const long long nch = pre[d.n_pop];
  for (int r = threadIdx.x; r < hist_rows; r += blockDim.x) cnt[r] = 0u;
  if (threadIdx.x == 0) {
    s_r0 = INT_MAX;
    s_r1 = -1;
    for (int q = 0; q < kScatterStages; ++q) mbar_init(&bar[q], 1);
    for (int q = 0; q < kScatterStages; ++q) {
      const long long c = blockIdx.x + (long long)q * gridDim.x;
      if (c < nch) scatter_issue(d, pre, sc, c, stages + (size_t)q * 5 * kScatterChunk, &bar[q]);
    }
  }
  __syncthreads();
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  Real* dstp[5] = {(Real*)d.y1, (Real*)d.y2, (Real*)d.yR, (Real*)d.yZ, (Real*)d.yT};
  long long local = 0;
  for (long long chunk = blockIdx.x; chunk < nch; chunk += gridDim.x, ++local) {
    const int q = (int)(local % kScatterStages);
    Real* st = stages + (size_t)q * 5 * kScatterChunk;
    const int pop = find_pop(pre, d.n_pop, chunk);
    const SortConst& P = sc[pop];
    const long long c0 = (chunk - pre[pop]) * kScatterChunk;
    if (!mbar_wait(&bar[q], (unsigned)((local / kScatterStages) & 1), d.err)) {
      // the later stages' copies in flight land before the CTA leaves
      if (threadIdx.x == 0)
        for (long long j = local + 1; j < local + kScatterStages && chunk + (j - local) * gridDim.x < nch; ++j)
          for (long long k = 0; k < (1ll << 22); ++k) {
            if (mbar_try_wait(&bar[j % kScatterStages], (unsigned)((j / kScatterStages) & 1))) break;
            __nanosleep(64);
          }
      return;
    }
    // the chunk's rows and their range
    int rows[kScatterItems];
    int lo = INT_MAX, hi = -1;
#pragma unroll
    for (int it = 0; it < kScatterItems; ++it) {
      const int j = it * kSortThreads + threadIdx.x;
      rows[it] = c0 + j < P.n ? sort_row(st[j], P.ih1, P.nrows) : -1;
      if (rows[it] >= 0) {
        lo = min(lo, rows[it]);
        hi = max(hi, rows[it]);
      }
    }
    lo = __reduce_min_sync(kFull, lo);
    hi = __reduce_max_sync(kFull, hi);
    if (lane == 0 && hi >= 0) {
      atomicMin(&s_r0, lo);
      atomicMax(&s_r1, hi);
    }
    __syncthreads();
    const int r1 = s_r1, r0 = r1 >= 0 ? s_r0 : 0;  // no live particle: the empty range [0, -1]
    const unsigned long long first = d.cell_off[P.cell_off];
    if (r0 == r1) {
#pragma unroll
      for (int it = 0; it < kScatterItems; ++it) {
        const unsigned m = __ballot_sync(kFull, rows[it] >= 0);
        if (lane == 0) s_wc[it * kSortWarps + w] = __popc(m);
      }
      __syncthreads();
      if (w == 0) {
        constexpr int kPer = kScatterItems * kSortWarps / 32;
        unsigned v[kPer], sum = 0;
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
          v[k] = s_wc[lane * kPer + k];
          sum += v[k];
        }
        unsigned incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const unsigned t = __shfl_up_sync(kFull, incl, o);
          if (lane >= o) incl += t;
        }
        unsigned ex = incl - sum;
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
          s_wc[lane * kPer + k] = ex;
          ex += v[k];
        }
        if (lane == 31)
          s_base = (unsigned)(d.cell_off[P.cell_off + r0] - first) + atomicAdd(d.cell_cnt + P.cell_off + r0, incl);
      }
      __syncthreads();
      const unsigned base = s_base, below = (1u << lane) - 1u;
#pragma unroll
      for (int it = 0; it < kScatterItems; ++it) {
        const unsigned m = __ballot_sync(kFull, rows[it] >= 0);
        if (rows[it] >= 0) {
          const int j = it * kSortThreads + threadIdx.x;
          const long long dst = P.base + (long long)(base + s_wc[it * kSortWarps + w] + __popc(m & below));
#pragma unroll
          for (int a = 0; a < 5; ++a) dstp[a][dst] = st[a * kScatterChunk + j];
        }
      }
    } else {
#pragma unroll
      for (int it = 0; it < kScatterItems; ++it) warp_count(cnt, rows[it]);
      __syncthreads();
      for (int r = r0 + threadIdx.x; r <= r1; r += blockDim.x) {
        const unsigned c = cnt[r];
        cur[r] = c ? (unsigned)(d.cell_off[P.cell_off + r] - first) + atomicAdd(d.cell_cnt + P.cell_off + r, c) : 0u;
      }
      __syncthreads();
#pragma unroll
      for (int it = 0; it < kScatterItems; ++it) {
        const unsigned pos = warp_count(cur, rows[it]);
        if (rows[it] >= 0) {
          const int j = it * kSortThreads + threadIdx.x;
          const long long dst = P.base + (long long)pos;
#pragma unroll
          for (int a = 0; a < 5; ++a) dstp[a][dst] = st[a * kScatterChunk + j];
        }
      }
      for (int r = r0 + threadIdx.x; r <= r1; r += blockDim.x) cnt[r] = 0u;
    }
    __syncthreads();  // the stage and the counters are free
    if (threadIdx.x == 0) {
      s_r0 = INT_MAX;
      s_r1 = -1;
      const long long nx = chunk + (long long)kScatterStages * gridDim.x;
      if (nx < nch) scatter_issue(d, pre, sc, nx, st, &bar[q]);
    }
  }
}

// Populations become dense: n = live particles, no freed slots.
__global__ void k_sort_finish(DevPtrs d) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= d.n_pop) return;
  const Pop& P = d.pop[p];
  d.ps[p].n = (long long)(d.cell_off[P.cell_off + P.cells] - d.cell_off[P.cell_off]);
  d.ps[p].n_holes = 0;
}

// Copy every slot [0, n) of one population to FP64 rows (dead slots keep
// their sentinel x1 > 0; the host drops them).
__global__ void k_copy_out(DevPtrs d, int pop, double* out, long long n) {
  long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  long long slot = d.pop[pop].base + k;
  out[5 * k + 0] = (double)((Real*)d.x1)[slot];
  out[5 * k + 1] = (double)((Real*)d.x2)[slot];
  out[5 * k + 2] = (double)((Real*)d.vR)[slot];
  out[5 * k + 3] = (double)((Real*)d.vZ)[slot];
  out[5 * k + 4] = (double)((Real*)d.vT)[slot];
}

unsigned blocks_for(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

}  // namespace

template <>
void launch_load<Real>(const DevPtrs& d, int pop, long long n0, long long count, long long draw0, int kind,
                       cudaStream_t s) {
  (void)kind;
  if (count <= 0) return;
  k_load<<<blocks_for(count, 256), 256, 0, s>>>(d, pop, n0, count, draw0);
}

template <>
void launch_explicit<Real>(const DevPtrs& d, int pop, long long n0, long long count, const double* dstate,
                           cudaStream_t s) {
  if (count <= 0) return;
  k_explicit<<<blocks_for(count, 256), 256, 0, s>>>(d, pop, n0, count, dstate);
}

template <>
void launch_deposit_all<Real>(const DevPtrs& d, int max_grid, int max_n2, cudaStream_t s) {
  const int win_n2 = max_n2 < kWinMaxN2 - 1 ? max_n2 : kWinMaxN2 - 1;
  const int sm = kWinRows * (win_n2 + 1) * (int)sizeof(unsigned long long);
  cudaFuncSetAttribute(k_deposit_all, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  k_deposit_all<<<max_grid, 256, sm, s>>>(d, win_n2);
}

// Dynamic shared memory of the push: window, chunk prefix, population constants.
// FP32 particles take the four-particle vector push (APIC_PUSH4=0: the
// one-particle push, for comparison).
static bool push4() {
  if (kF64) return false;
  static int on = -1;
  if (on < 0) {
    const char* e = std::getenv("APIC_PUSH4");
    on = e ? (std::atoi(e) != 0) : 1;
  }
  return on != 0;
}

static int push_smem(int rows, int win_n2, int n_pop) {
  const int words = kF64 ? rows * (win_n2 + 1) : 2 * rows * win_n2;
  return words * (int)sizeof(unsigned long long) + (n_pop + 1) * (int)sizeof(long long) +
         n_pop * (int)sizeof(PushConst);
}

template <>
int push_window_rows<Real>(int max_n2) {
  // window capacity: the widest grid of the batch, up to kWinMaxN2 - 1 cells
  // (wider grids deposit straight to global memory); node rows up to
  // kWinRows within 48 KB (a 512-cell row of FP32 cell moments takes 8 KB;
  // on the 1024 x 512 grid with 1e8 particles the vector push took 1.55 ms
  // with 4 rows, 1.47 with 6, 1.51 with 8, 1.75 with 10: wider windows leave
  // less L1 to the gather) and as many as keep the push's CTAs per SM
  // resident.  Cached per width: the first call (at set-up, before any
  // capture) queries the occupancy.  apic_autotune tries 2 to 16 rows.
  const int win_n2 = max_n2 < kWinMaxN2 - 1 ? max_n2 : kWinMaxN2 - 1;
  static int rows_for[kWinMaxN2 + 1] = {};
  int rows = rows_for[win_n2];
  if (rows == 0) {
    const int row_bytes = (kF64 ? (win_n2 + 1) : 2 * win_n2) * (int)sizeof(unsigned long long);
    rows = std::max(2, std::min(kWinRows, 49152 / std::max(1, row_bytes)));
    const char* e = std::getenv("APIC_WIN_ROWS");  // tuning: a fixed row count
    if (e) rows = std::max(2, std::min(kPushWinRows, std::atoi(e)));
    const void* kern = push4() ? (const void*)k_push4<false> : (const void*)k_push<false>;
    const int want = push4() ? (int)APIC_PUSH4_MIN_BLOCKS : (int)APIC_PUSH_MIN_BLOCKS;
    for (; !e && rows > 2; --rows) {
      const int sm = push_smem(rows, win_n2, kMaxPop);
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
      int per = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, 256, sm) == cudaSuccess && per >= want) break;
    }
    cudaGetLastError();
    rows_for[win_n2] = rows;
  }
  return rows;
}

template <>
void launch_push<Real>(const DevPtrs& d, int grid, int max_n2, bool chord, int win_rows, int chunk_group,
                       int chunk_items, long long particles, cudaStream_t s) {
  const int win_n2 = max_n2 < kWinMaxN2 - 1 ? max_n2 : kWinMaxN2 - 1;
  const int rows = win_rows > 0 ? std::max(2, std::min(kPushWinRows, win_rows)) : push_window_rows<Real>(max_n2);
  const int sm = push_smem(rows, win_n2, d.n_pop);
  const bool v4 = push4();
  const void* kern = v4 ? (chord ? (const void*)k_push4<true> : (const void*)k_push4<false>)
                        : (chord ? (const void*)k_push<true> : (const void*)k_push<false>);
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  static int group_env = -1;  // chunks per group (APIC_PUSH_GROUP, default 4: the fastest of 1, 2, 4, 8 measured)
  if (group_env < 0) {
    const char* e = std::getenv("APIC_PUSH_GROUP");
    group_env = e ? std::max(1, std::atoi(e)) : 4;
  }
  const int group = chunk_group > 0 ? chunk_group : group_env;
  cudaMemsetAsync(d.cnt + 1, 0, sizeof(long long), s);  // the group counter
  if (v4) {
    grid = std::max(1, grid / 4 * (int)APIC_PUSH4_MIN_BLOCKS);  // the caller's grid is 4 CTAs per SM
    // 8192-particle chunks when every CTA still gets two dozen of them
    int ci = chunk_items == 16 || chunk_items == 32 ? chunk_items
                                                    : (particles >= 24ll * 8192 * grid ? kPush4ItemsMax : 16);
    if (chord) k_push4<true><<<grid, 256, sm, s>>>(d, win_n2, rows, group, ci);
    else k_push4<false><<<grid, 256, sm, s>>>(d, win_n2, rows, group, ci);
  } else if (chord) {
    k_push<true><<<grid, 256, sm, s>>>(d, win_n2, rows, group);
  } else {
    k_push<false><<<grid, 256, sm, s>>>(d, win_n2, rows, group);
  }
}

template <>
void launch_inject<Real>(const DevPtrs& d, long long max_inj, cudaStream_t s) {
  if (max_inj <= 0) return;
  // few CTAs, several injections per thread: fewer window flushes
  unsigned gx = blocks_for(max_inj, 256);
  gx = gx < 160 ? gx : 160;
  dim3 g(gx, d.n_pop);
  k_inject<<<g, 256, 0, s>>>(d);
}

// Resident CTAs per SM of the two sort passes for grids of up to `rows` cell
// rows (their dynamic shared memory grows with the rows), from the occupancy
// calculator, cached per row count.
static int s_sort_ctas[2][4097] = {};

static int count_smem(int hist_rows) { return hist_rows * (int)sizeof(unsigned); }

template <>
void sort_setup<Real>(int max_rows) {
  max_rows = std::max(1, std::min(4096, max_rows));
  if (s_sort_ctas[0][max_rows] > 0) return;
  const void* kern[2] = {(const void*)k_sort_count, (const void*)k_sort_scatter};
  const int smem[2] = {count_smem(max_rows), scatter_smem(max_rows)};
  const int most[2] = {8, 4};
  for (int k = 0; k < 2; ++k) {
    // the limit for the largest grid, so that every simulation's launches fit it
    cudaFuncSetAttribute(kern[k], cudaFuncAttributeMaxDynamicSharedMemorySize, k ? scatter_smem(4096) : count_smem(4096));
    int per = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern[k], kSortThreads, smem[k]) != cudaSuccess) per = 1;
    s_sort_ctas[k][max_rows] = std::max(1, std::min(most[k], per));
  }
  cudaGetLastError();
}

template <>
void launch_sort<Real>(const DevPtrs& d, int grid, int max_rows, cudaStream_t s) {
  const int sms = std::max(1, grid / 4);  // the caller's grid is 4 CTAs per SM
  max_rows = std::max(1, std::min(4096, max_rows));
  sort_setup<Real>(max_rows);
  cudaMemsetAsync(d.cell_cnt, 0, sizeof(unsigned) * d.total_cells, s);
  k_sort_count<<<sms * s_sort_ctas[0][max_rows], kSortThreads, count_smem(max_rows), s>>>(d, max_rows);
  int nb = (int)((d.total_cells + 1023) / 1024);
  k_scan_blocks<<<nb, 1024, 0, s>>>(d);
  k_scan_top<<<1, 1024, 0, s>>>(d, nb);
  k_scan_add<<<nb, 1024, 0, s>>>(d);
  k_sort_scatter<<<sms * s_sort_ctas[1][max_rows], kSortThreads, scatter_smem(max_rows), s>>>(d, max_rows);
  k_sort_finish<<<(d.n_pop + 63) / 64, 64, 0, s>>>(d);
}

template <>
void launch_gather_particles<Real>(const DevPtrs& d, int pop, double* out, long long* n_out, cudaStream_t s) {
  long long n = *n_out;
  if (n <= 0) return;
  k_copy_out<<<blocks_for(n, 256), 256, 0, s>>>(d, pop, out, n);
}

}  // namespace apic
