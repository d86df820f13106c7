// Reverse sweep (adjoint) of a K-step window of the APIC step
// (arXiv:2307.11107, Secs. 1-2): the gradient of L = sum_o dL/dout_o out_o
// (window means of drag F_Z, electric F_Z, current, torque T_z and grain
// charge Q) with respect to the grain shape alpha (Eqs. 2-5, 7), the grain
// potential phi_g (boundary value of Eq. 6) and the axial field B (Eq. 9), at
// fixed decisions (absorbed, escaped or kept, injection counts, cells): the
// transpose of the forward-mode window's Jacobian, computed backwards.
//
// Forward pass (the ordinary step, with per-step checkpoints): the particle
// state at the start of each step, rho and phi, each slot's fate in the push
// and each injection draw's slot.  Reverse pass, step K-1 down to 0, in the
// reverse order of the step:
//   injection   the adjoint of an injected particle's state times its
//               alpha-derivative (Eq. 4 sampling at the same random numbers);
//   push        per particle, the transpose of its local Jacobian (the step's
//               gather of Eq. 10, Boris push of Eq. 9, chord, rotation and
//               Eq. 2, or the tallies of an absorbed particle) applied to its
//               adjoint; the local Jacobian comes from dual numbers, three
//               directions at a time (state, gathered field, alpha, B);
//   surface     the seeds of the electric force and grain charge on phi;
//   gradients   the transpose of the node differences;
//   Poisson     lambda_b = A^-T lambda_phi with the nested-dissection fronts
//               of A applied transposed (FP64), and the terms of phi_g (the
//               Dirichlet row) and alpha (the operator's derivative);
//   deposit     the transpose of the bilinear weighing onto the particles and
//               the alpha-derivative of w = V_domain / N and of the volumes.
//
// Compiled once per particle precision (-DAPIC_REAL=double | float); the
// node-side kernels only in the double build (APIC_ADJOINT_COMMON).
#include <cuda_runtime.h>

#include <cstdint>

#include "apic_internal.h"
#include "dual.cuh"
#include "geom.cuh"

#ifndef APIC_REAL
#error "compile with -DAPIC_REAL=float or -DAPIC_REAL=double"
#endif

namespace apic {
namespace {

#include "particle_common.cuh"

using Real2 = typename Pair<Real>::T;
template <int N>
using DN = ad::Dual<Real, N>;
using D3 = DN<3>;
using D1 = DN<1>;

__device__ __forceinline__ Real val(Real x) { return x; }
template <int N>
__device__ __forceinline__ Real val(const ad::Dual<Real, N>& x) {
  return x.v;
}

__device__ __forceinline__ const Real* ckc(const AdjPtrs& a, int k, int c) {
  return (const Real*)a.ck + ((long long)k * 5 + c) * a.stride;
}

// Prefix of the populations' slot counts at the start of step k (one thread).
__device__ __forceinline__ void pop_prefix_at(const DevPtrs& d, const PopState* ps, long long* pre) {
  if (threadIdx.x == 0) {
    long long s = 0;
    for (int p = 0; p < d.n_pop; ++p) {
      pre[p] = s;
      s += ps[p].n;
    }
    pre[d.n_pop] = s;
  }
  __syncthreads();
}

// One particle's push in number type T, the same sequence as the step's push
// (gather of Eq. 10 with the bilinear weights of the cell the values give,
// Boris push with the field vector -B z-hat, straight chord, rotation back to
// the meridional plane, Eq. 2).  dg1, dg2 are added to the gathered node
// gradients (zero: their directions carry the field's adjoint).
template <class T>
struct PushIO {
  T x1n, x2n, vRn, vz, vTn;  // the new state of a kept particle
  T R, Z, vx, vy;            // chord start and the velocity at n + 1/2 (tallies)
  Real w[4];                 // gather weights (values) of the corners below
  long long n[4];
  bool hit, out;
};

template <class T>
__device__ __forceinline__ void push_eval(const Inst& I, const Real2* G, T x1, T x2, T vR, T vZ, T vT, T dg1, T dg2,
                                          T al, T B, Real h, PushIO<T>& o) {
  const Real dt = (Real)I.dt;
  T r = radius(al, x1, x2);
  T sn = sqrt((Real(1) - x2) * (Real(1) + x2));
  T R = r * sn, Z = r * x2;
  T u1 = (x1 + Real(1)) / (Real)I.h1;
  T u2 = (x2 + Real(1)) / (Real)I.h2;
  int ci = (int)floor(val(u1)), cj = (int)floor(val(u2));
  ci = ci < 0 ? 0 : (ci > I.n1 - 1 ? I.n1 - 1 : ci);
  cj = cj < 0 ? 0 : (cj > I.n2 - 1 ? I.n2 - 1 : cj);
  T f1 = u1 - (Real)ci, f2 = u2 - (Real)cj;
  if (val(f1) < Real(0)) f1 = T(Real(0));
  if (val(f1) > Real(1)) f1 = T(Real(1));
  if (val(f2) < Real(0)) f2 = T(Real(0));
  if (val(f2) > Real(1)) f2 = T(Real(1));
  const long long n00 = I.node_off + (long long)ci * I.N2 + cj;
  o.n[0] = n00;
  o.n[1] = n00 + I.N2;
  o.n[2] = n00 + 1;
  o.n[3] = n00 + I.N2 + 1;
  const Real2 a00 = G[o.n[0]], a10 = G[o.n[1]], a01 = G[o.n[2]], a11 = G[o.n[3]];
  T w00 = (Real(1) - f1) * (Real(1) - f2), w10 = f1 * (Real(1) - f2);
  T w01 = (Real(1) - f1) * f2, w11 = f1 * f2;
  o.w[0] = val(w00);
  o.w[1] = val(w10);
  o.w[2] = val(w01);
  o.w[3] = val(w11);
  T g1 = w00 * a00.x + w10 * a10.x + w01 * a01.x + w11 * a11.x + dg1;
  T g2 = w00 * a00.y + w10 * a10.y + w01 * a01.y + w11 * a11.y + dg2;
  Metric<T> m = metric(al, r, x2);
  T ER = -(m.x1R * g1 + m.x2R * g2);
  T EZ = -(m.x1Z * g1 + m.x2Z * g2);
  T vx = vR + h * ER, vy = vT, vz = vZ + h * EZ;
  T tz = h * (-B);
  T sz = Real(2) * tz / (Real(1) + tz * tz);
  T px_ = vx + vy * tz, py_ = vy - vx * tz;
  vx = vx + py_ * sz;
  vy = vy - px_ * sz;
  vx = vx + h * ER;
  vz = vz + h * EZ;
  T Xc = R + vx * dt, Yc = vy * dt, Zn = Z + vz * dt;
  T Rn = sqrt(Xc * Xc + Yc * Yc);
  T cr(Real(1)), sr(Real(0));
  if (val(Rn) > Real(0)) {
    cr = Xc / Rn;
    sr = Yc / Rn;
  }
  o.vRn = cr * vx + sr * vy;
  o.vTn = -sr * vx + cr * vy;
  T rn = sqrt(Rn * Rn + Zn * Zn);
  o.x2n = Zn / rn;
  o.hit = val(rn) < r_grain(val(al), val(o.x2n));
  o.x1n = x1_at(al, rn, o.x2n);
  o.out = !o.hit && val(o.x1n) > (Real)I.x1_out;
  o.vz = vz;
  o.R = R;
  o.Z = Z;
  o.vx = vx;
  o.vy = vy;
}

// ---- forward pass ----
// The step's push (values), each slot's fate recorded: 0 kept, 1 absorbed,
// 2 escaped, 3 no live particle.
__global__ void __launch_bounds__(256) k_adj_fwd_push(DevPtrs d, AdjPtrs a, int k) {
  __shared__ long long s_pre[kMaxPop + 1];
  pop_prefix_at(d, d.ps, s_pre);
  const long long total = s_pre[d.n_pop];
  const Real2* G = (const Real2*)d.G;
  uint8_t* fate = a.fate + (long long)k * a.stride;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < total;
       q += (long long)gridDim.x * blockDim.x) {
    const int pop = find_pop(s_pre, d.n_pop, q);
    const Pop& P = d.pop[pop];
    const Inst& I = d.inst[P.inst];
    const long long kk = q - s_pre[pop], slot = P.base + kk;
    const Real x1 = ((const Real*)d.x1)[slot];
    if (!(x1 < Real(0))) {
      fate[slot] = 3;
      continue;
    }
    PushIO<Real> o;
    const Real h = Real(0.5) * (Real)(P.q / P.m) * (Real)I.dt;
    push_eval<Real>(I, G, x1, ((const Real*)d.x2)[slot], ((const Real*)d.vR)[slot], ((const Real*)d.vZ)[slot],
                    ((const Real*)d.vT)[slot], Real(0), Real(0), (Real)I.alpha, (Real)I.B, h, o);
    if (o.hit) {
      absorb_tally(d, I, P, o.R, o.Z, o.vx, o.vz, o.vy, (Real)I.dt);
      atomicAdd((unsigned long long*)&d.ps[pop].absorbed, 1ull);
      ((Real*)d.x1)[slot] = Real(2);
      push_hole(d, P, pop, kk);
      fate[slot] = 1;
      continue;
    }
    if (o.out) {
      atomicAdd((unsigned long long*)&d.ps[pop].escaped, 1ull);
      ((Real*)d.x1)[slot] = Real(2);
      push_hole(d, P, pop, kk);
      fate[slot] = 2;
      continue;
    }
    ((Real*)d.x1)[slot] = o.x1n;
    ((Real*)d.x2)[slot] = o.x2n;
    ((Real*)d.vR)[slot] = o.vRn;
    ((Real*)d.vZ)[slot] = o.vz;
    ((Real*)d.vT)[slot] = o.vTn;
    fate[slot] = 0;
  }
}

// An injected particle's state (values and alpha-derivative) from its draws:
// x2 from the inverse CDF of Eq. 4 on x1_out (its alpha-derivative from the
// table's), a flux-weighted half-Maxwellian along -grad x1 and Maxwellian
// tangential and Theta components, a free flight of a uniform fraction of dt.
struct Inj {
  D1 x1n, x2n, vRn, vz, vTn;  // stored state
  D1 R, Z, vx, vy;            // flight start and velocity (tallies)
  Real tau;
  bool hit, out;
};

__device__ __forceinline__ void inject_eval(const DevPtrs& d, const TanPtrs& t, const Inst& I, const Pop& P,
                                            long long g, Inj& o) {
  uint32_t u[8];
  draws8(I, P, g, 2u, u);
  const D1 al = D1::seed((Real)I.alpha, 0);
  const Real dt = (Real)I.dt;
  const double* cdf = d.tab + I.tab_off + (kTable + 1);
  const double* dcdf = t.dtab + I.tab_off + (kTable + 1);
  const Real u0 = unit(u[0]);
  const double tq = (double)u0 * cdf[kTable];
  const int lo = table_interval(cdf, d.guide + I.tab_off + (kTable + 1), (double)u0, tq);
  const double dlt = cdf[lo + 1] - cdf[lo];
  const double f = dlt > 0.0 ? (tq - cdf[lo]) / dlt : 0.5;
  const double ht = 2.0 / kTable;
  const double dtq = (double)u0 * dcdf[kTable];
  const double df = dlt > 0.0 ? (dtq - dcdf[lo] - f * (dcdf[lo + 1] - dcdf[lo])) / dlt : 0.0;
  D1 x2((Real)(-1.0 + lo * ht + f * ht));
  x2.d[0] = (Real)(df * ht);
  const Real vth = (Real)P.vth;
  const Real vn = vth * sqrt(Real(-2) * log(unit(u[1])));
  const Real ra = sqrt(Real(-2) * log(unit(u[2])));
  const Real pa = Real(2 * kPi) * unit(u[3]);
  const Real vt = vth * (ra * cos(pa)), vth_ = vth * (ra * sin(pa));
  o.tau = unit(u[4]) * dt;
  D1 r = radius(al, D1((Real)I.x1_out), x2);
  D1 sn = sqrt((Real(1) - x2) * (Real(1) + x2));
  o.R = r * sn;
  o.Z = r * x2;
  Metric<D1> m = metric(al, r, x2);
  D1 gn = sqrt(m.x1R * m.x1R + m.x1Z * m.x1Z);
  D1 nR = -m.x1R / gn, nZ = -m.x1Z / gn;
  D1 tR = nZ, tZ = -nR;
  o.vx = vn * nR + vt * tR;
  o.vz = vn * nZ + vt * tZ;
  o.vy = D1(vth_);
  D1 Xc = o.R + o.vx * o.tau, Yc = o.vy * o.tau, Zn = o.Z + o.vz * o.tau;
  D1 Rn = sqrt(Xc * Xc + Yc * Yc);
  D1 cr(Real(1)), sr(Real(0));
  if (Rn.v > Real(0)) {
    cr = Xc / Rn;
    sr = Yc / Rn;
  }
  D1 rn = sqrt(Rn * Rn + Zn * Zn);
  o.x2n = Zn / rn;
  o.hit = rn.v < r_grain(al.v, o.x2n.v);
  o.x1n = x1_at(al, rn, o.x2n);
  o.out = !o.hit && o.x1n.v > (Real)I.x1_out;
  o.vRn = cr * o.vx + sr * o.vy;
  o.vTn = -sr * o.vx + cr * o.vy;
}

// The step's surface injection (values), each draw's slot recorded (from the
// population's base; -1 absorbed in its first flight, -2 escaped).
__global__ void __launch_bounds__(256) k_adj_fwd_inject(DevPtrs d, AdjPtrs a, TanPtrs t, int k) {
  const int pop = blockIdx.y;
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  PopState& S = d.ps[pop];
  const Pop& P = d.pop[pop];
  const Inst& I = d.inst[P.inst];
  if (q >= S.n_inj) return;
  int64_t* rec = a.inj + ((long long)k * d.n_pop + pop) * a.inj_cap;
  Inj o;
  inject_eval(d, t, I, P, S.draws + q, o);
  if (o.hit) {
    absorb_tally(d, I, P, o.R.v, o.Z.v, o.vx.v, o.vz.v, o.vy.v, o.tau);
    atomicAdd((unsigned long long*)&S.absorbed, 1ull);
    if (q < a.inj_cap) rec[q] = -1;
    return;
  }
  if (o.out) {
    atomicAdd((unsigned long long*)&S.escaped, 1ull);
    if (q < a.inj_cap) rec[q] = -2;
    return;
  }
  const long long sidx = (long long)atomicAdd((unsigned long long*)&S.inj_stored, 1ull);
  const long long nh = S.n_holes, n = S.n;
  const long long kk = sidx < nh ? d.holes[P.base + nh - 1 - sidx] : n + (sidx - nh);
  if (kk >= P.cap) {
    atomicAdd((unsigned long long*)&S.dropped, 1ull);
    atomicOr(d.err, kErrCapacity);
    if (q < a.inj_cap) rec[q] = -2;
    return;
  }
  const long long slot = P.base + kk;
  ((Real*)d.x1)[slot] = o.x1n.v;
  ((Real*)d.x2)[slot] = o.x2n.v;
  ((Real*)d.vR)[slot] = o.vRn.v;
  ((Real*)d.vZ)[slot] = o.vz.v;
  ((Real*)d.vT)[slot] = o.vTn.v;
  if (q < a.inj_cap) rec[q] = kk;
}

// ---- reverse pass ----
// Parameter adjoints of one thread (instance inst) added to the instance's
// totals: a warp whose lanes share the instance adds its sum once.
__device__ __forceinline__ void add_grad(const AdjPtrs& a, int inst, double ga, double gp, double gb) {
  const unsigned full = 0xffffffffu;
  const int i0 = __shfl_sync(full, inst, 0);
  if (__all_sync(full, inst == i0)) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      ga += __shfl_down_sync(full, ga, o);
      gp += __shfl_down_sync(full, gp, o);
      gb += __shfl_down_sync(full, gb, o);
    }
    if ((threadIdx.x & 31) == 0 && i0 >= 0) {
      if (ga != 0.0) atomicAdd(a.grad + i0 * kNPar + 0, ga);
      if (gp != 0.0) atomicAdd(a.grad + i0 * kNPar + 1, gp);
      if (gb != 0.0) atomicAdd(a.grad + i0 * kNPar + 2, gb);
    }
  } else if (inst >= 0) {
    if (ga != 0.0) atomicAdd(a.grad + inst * kNPar + 0, ga);
    if (gp != 0.0) atomicAdd(a.grad + inst * kNPar + 1, gp);
    if (gb != 0.0) atomicAdd(a.grad + inst * kNPar + 2, gb);
  }
}

// Injection of step k backwards: a stored particle's adjoint (from the later
// steps) times its state's alpha-derivative, and the slot's adjoint cleared
// (before the step's injection it held no particle, or one that left in
// this step's push); a particle absorbed in its first flight adds its
// tallies' alpha-derivatives (w = V_domain / N moves with alpha too).
__global__ void __launch_bounds__(256) k_adj_rev_inject(DevPtrs d, AdjPtrs a, TanPtrs t, int k) {
  const int pop = blockIdx.y;
  const Pop& P = d.pop[pop];
  const Inst& I = d.inst[P.inst];
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long g0 = a.ck_ps[(long long)k * d.n_pop + pop].draws;
  const long long n_inj = a.ck_ps[(long long)(k + 1) * d.n_pop + pop].draws - g0;
  double ga = 0.0;
  int inst = -1;
  if (q < n_inj && q < a.inj_cap) {
    const int64_t rec = a.inj[((long long)k * d.n_pop + pop) * a.inj_cap + q];
    if (rec != -2) {
      inst = P.inst;
      Inj o;
      inject_eval(d, t, I, P, g0 + q, o);
      if (rec >= 0) {
        const long long slot = P.base + rec;
        double* L = a.lam;
        const D1* st[5] = {&o.x1n, &o.x2n, &o.vRn, &o.vz, &o.vTn};
#pragma unroll
        for (int c = 0; c < 5; ++c) {
          ga += L[(long long)c * a.stride + slot] * (double)st[c]->d[0];
          L[(long long)c * a.stride + slot] = 0.0;
        }
      } else {
        const double* sd = a.seed + (long long)P.inst * kNOut;
        const double dt = I.dt, w = P.w, dl = t.dlnw[P.inst];
        const double vz = o.vz.v, Rvy = (double)o.R.v * o.vy.v;
        const double dvz = o.vz.d[0], dRvy = (double)o.R.d[0] * o.vy.v + (double)o.R.v * o.vy.d[0];
        ga += sd[0] / dt * P.m * w * (dvz + vz * dl) + sd[3] / dt * P.m * w * (dRvy + Rvy * dl) +
              sd[2] / dt * P.q * w * dl;
      }
    }
  }
  add_grad(a, inst, ga, 0.0, 0.0);
}

// Push of step k backwards.  For each slot live at the start of the step
// (the checkpoint), the transpose of the particle's local Jacobian applied to
// the adjoint of its push's result: the new state's adjoint for a kept
// particle, the output seeds of its tallies for an absorbed one, nothing for
// an escaped one.  The local Jacobian comes from push_eval on three-direction
// duals in three passes: (x1, x2, vR), (vZ, vTheta, g1), (g2, alpha, B).
// The slot's adjoint becomes that of its state at the start of the step; the
// gathered field's adjoint goes to the four corner nodes with the bilinear
// weights.
__global__ void __launch_bounds__(256) k_adj_rev_push(DevPtrs d, AdjPtrs a, TanPtrs t, int k) {
  __shared__ long long s_pre[kMaxPop + 1];
  const PopState* ps = a.ck_ps + (long long)k * d.n_pop;
  pop_prefix_at(d, ps, s_pre);
  const long long total = s_pre[d.n_pop];
  const Real2* G = (const Real2*)a.Gk;
  const uint8_t* fate = a.fate + (long long)k * a.stride;
  const long long tn = d.total_nodes;
  for (long long q0 = (long long)blockIdx.x * blockDim.x; q0 < total; q0 += (long long)gridDim.x * blockDim.x) {
    const long long q = q0 + threadIdx.x;
    double ga = 0.0, gb = 0.0;
    int inst = -1;
    if (q < total) {
      const int pop = find_pop(s_pre, d.n_pop, q);
      const Pop& P = d.pop[pop];
      const Inst& I = d.inst[P.inst];
      const long long slot = P.base + (q - s_pre[pop]);
      const int f = fate[slot];
      double* L = a.lam;
      if (f == 0 || f == 1) {
        inst = P.inst;
        double lout[5];
#pragma unroll
        for (int c = 0; c < 5; ++c) lout[c] = f == 0 ? L[(long long)c * a.stride + slot] : 0.0;
        const double* sd = a.seed + (long long)P.inst * kNOut;
        const double dt = I.dt, w = P.w, dl = t.dlnw[P.inst];
        const Real xs[5] = {ckc(a, k, 0)[slot], ckc(a, k, 1)[slot], ckc(a, k, 2)[slot], ckc(a, k, 3)[slot],
                            ckc(a, k, 4)[slot]};
        const Real h = Real(0.5) * (Real)(P.q / P.m) * (Real)I.dt;
        double lin[9];
        Real wts[4];
        long long nodes[4];
#pragma unroll 1
        for (int pass = 0; pass < 3; ++pass) {
          D3 in[9];
#pragma unroll
          for (int z = 0; z < 9; ++z) {
            const Real v = z < 5 ? xs[z] : (z == 7 ? (Real)I.alpha : (z == 8 ? (Real)I.B : Real(0)));
            in[z] = (z / 3 == pass) ? D3::seed(v, z % 3) : D3(v);
          }
          PushIO<D3> o;
          push_eval<D3>(I, G, in[0], in[1], in[2], in[3], in[4], in[5], in[6], in[7], in[8], h, o);
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            wts[c] = o.w[c];
            nodes[c] = o.n[c];
          }
#pragma unroll
          for (int e = 0; e < 3; ++e) {
            const int z = 3 * pass + e;
            double acc;
            if (f == 0) {
              acc = lout[0] * (double)o.x1n.d[e] + lout[1] * (double)o.x2n.d[e] + lout[2] * (double)o.vRn.d[e] +
                    lout[3] * (double)o.vz.d[e] + lout[4] * (double)o.vTn.d[e];
            } else {
              const double Rvy = (double)o.R.v * o.vy.v;
              const double dRvy = (double)o.R.d[e] * o.vy.v + (double)o.R.v * o.vy.d[e];
              const double a_w = z == 7 ? dl : 0.0;  // w moves with alpha
              acc = sd[0] / dt * P.m * w * ((double)o.vz.d[e] + (double)o.vz.v * a_w) +
                    sd[3] / dt * P.m * w * (dRvy + Rvy * a_w) + sd[2] / dt * P.q * w * a_w;
            }
            lin[z] = acc;
          }
        }
#pragma unroll
        for (int c = 0; c < 5; ++c) L[(long long)c * a.stride + slot] = lin[c];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          if (wts[c] == Real(0)) continue;
          atomicAdd(a.lG + nodes[c], (double)wts[c] * lin[5]);
          atomicAdd(a.lG + tn + nodes[c], (double)wts[c] * lin[6]);
        }
        ga = lin[7];
        gb = lin[8];
      } else {
#pragma unroll
        for (int c = 0; c < 5; ++c) L[(long long)c * a.stride + slot] = 0.0;
      }
    }
    add_grad(a, inst, ga, 0.0, gb);
  }
}

// Deposit of step k backwards: rho = sum_p q w S(x_p) / V, so the adjoint of
// a live particle's (x1, x2) gains q w sum_c (dS_c / dx) lambda_rho_c / V_c
// (bilinear weights of its cell; a clamped fraction carries none).
__global__ void __launch_bounds__(256) k_adj_rev_deposit(DevPtrs d, AdjPtrs a, int k) {
  __shared__ long long s_pre[kMaxPop + 1];
  const PopState* ps = a.ck_ps + (long long)k * d.n_pop;
  pop_prefix_at(d, ps, s_pre);
  const long long total = s_pre[d.n_pop];
  const uint8_t* fate = a.fate + (long long)k * a.stride;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < total;
       q += (long long)gridDim.x * blockDim.x) {
    const int pop = find_pop(s_pre, d.n_pop, q);
    const Pop& P = d.pop[pop];
    const Inst& I = d.inst[P.inst];
    const long long slot = P.base + (q - s_pre[pop]);
    if (fate[slot] == 3) continue;
    const double x1 = (double)ckc(a, k, 0)[slot], x2 = (double)ckc(a, k, 1)[slot];
    const double u1 = (x1 + 1.0) / I.h1, u2 = (x2 + 1.0) / I.h2;
    int ci = (int)floor(u1), cj = (int)floor(u2);
    ci = ci < 0 ? 0 : (ci > I.n1 - 1 ? I.n1 - 1 : ci);
    cj = cj < 0 ? 0 : (cj > I.n2 - 1 ? I.n2 - 1 : cj);
    double f1 = u1 - ci, f2 = u2 - cj, d1 = 1.0 / I.h1, d2 = 1.0 / I.h2;
    if (f1 < 0.0 || f1 > 1.0) {
      f1 = f1 < 0.0 ? 0.0 : 1.0;
      d1 = 0.0;
    }
    if (f2 < 0.0 || f2 > 1.0) {
      f2 = f2 < 0.0 ? 0.0 : 1.0;
      d2 = 0.0;
    }
    const long long n00 = I.node_off + (long long)ci * I.N2 + cj;
    const long long nn[4] = {n00, n00 + I.N2, n00 + 1, n00 + I.N2 + 1};
    double l[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) l[c] = a.lrho[nn[c]] / d.V[nn[c]];
    // dS/dx1 = d1 (-(1 - f2), (1 - f2), -f2, f2); dS/dx2 = d2 (-(1 - f1), -f1, (1 - f1), f1)
    const double qw = P.q * P.w;
    const double gx1 = d1 * (-(1.0 - f2) * l[0] + (1.0 - f2) * l[1] - f2 * l[2] + f2 * l[3]);
    const double gx2 = d2 * (-(1.0 - f1) * l[0] - f1 * l[1] + (1.0 - f1) * l[2] + f1 * l[3]);
    a.lam[slot] += qw * gx1;
    a.lam[a.stride + slot] += qw * gx2;
  }
}

#ifdef APIC_ADJOINT_COMMON
__device__ __forceinline__ double x2_node(const Inst& I, int j) { return j == I.n2 ? 1.0 : -1.0 + j * I.h2; }

// Deterministic block sum (fixed tree) of one double per thread; blockDim 256.
__device__ double block_sum(double v, double* sh) {
  int t = threadIdx.x;
  sh[t] = v;
  __syncthreads();
  for (int o = blockDim.x >> 1; o > 0; o >>= 1) {
    if (t < o) sh[t] += sh[t + o];
    __syncthreads();
  }
  double r = sh[0];
  __syncthreads();
  return r;
}

// Window sums of the step's outputs (before the step's bookkeeping clears the
// step tallies).
__global__ void k_adj_values(DevPtrs d, AdjPtrs a) {
  const int inst = blockIdx.x * blockDim.x + threadIdx.x;
  if (inst >= d.n_inst) return;
  const Inst& I = d.inst[inst];
  const StepState& T = d.stp[inst];
  double tl[5];
  step_tallies(d, inst, tl);
  double* v = a.vals + (long long)inst * kNOut;
  v[0] += tl[1] / I.dt;
  v[1] += T.FZ;
  v[2] += tl[0] / I.dt;
  v[3] += tl[2] / I.dt;
  v[4] += T.Q;
}

// Seeds of the electric force and grain charge of step k on phi (rows 0..2
// through the one-sided dphi/dx1 on the grain), and their alpha-derivative at
// fixed phi (|grad x1|, n_Z and dA of Eq. 4 on the grain).
__global__ void __launch_bounds__(256) k_adj_surface(DevPtrs d, AdjPtrs a, TanPtrs t, int k) {
  __shared__ double sh[256];
  const int inst = blockIdx.x;
  const Inst& I = d.inst[inst];
  const bool nofield = (I.flags & APIC_NO_FIELD) != 0;
  const int N2 = I.N2;
  const double* p0 = a.ck_phi + (long long)k * d.total_nodes + I.node_off;
  const double sF = a.seed[(long long)inst * kNOut + 1], sQ = a.seed[(long long)inst * kNOut + 4];
  double ga = 0.0;
  for (int j = threadIdx.x; j <= I.n2 && !nofield; j += blockDim.x) {
    using DD = ad::Dual<double, 1>;
    const double x2 = x2_node(I, j);
    DD al = DD::seed(I.alpha, 0), X2(x2);
    DD r = r_grain(al, X2);
    Metric<DD> m = metric(al, r, X2);
    DD g = sqrt(m.x1R * m.x1R + m.x1Z * m.x1Z);
    DD dA = area_density(al, DD(-1.0), X2);
    DD nzda = (m.x1Z / g) * dA;
    const double G1 = (-3.0 * p0[j] + 4.0 * p0[N2 + j] - p0[2 * N2 + j]) / (2.0 * I.h1);
    const double En = -G1 * g.v;
    const double tw = (j == 0 || j == I.n2) ? 0.5 * I.h2 : I.h2;
    // dL/dE_n and the E_n derivative along alpha at fixed phi
    const double dLdE = sQ * tw * dA.v + sF * tw * En * nzda.v;
    const double dEa = -G1 * g.d[0];
    ga += dLdE * dEa + sQ * tw * En * dA.d[0] + sF * tw * 0.5 * En * En * nzda.d[0];
    const double c = -g.v / (2.0 * I.h1);  // dE_n / dphi = c (-3, 4, -1) on rows 0, 1, 2
    double* lp = a.lphi + I.node_off;
    lp[j] += dLdE * c * -3.0;
    lp[N2 + j] += dLdE * c * 4.0;
    lp[2 * N2 + j] += dLdE * c * -1.0;
  }
  const double tot = block_sum(ga, sh);
  if (threadIdx.x == 0 && tot != 0.0) atomicAdd(a.grad + (long long)inst * kNPar + 0, tot);
}

// lambda_phi += D^T lambda_G: the transpose of the node gradients (central
// differences inside, one-sided second order on the four edges).
__global__ void __launch_bounds__(256) k_adj_gradT(DevPtrs d, AdjPtrs a) {
  const Inst& I = d.inst[blockIdx.y];
  const int n1 = I.n1, n2 = I.n2, N2 = I.N2;
  const double* l1 = a.lG + I.node_off;
  const double* l2 = a.lG + d.total_nodes + I.node_off;
  const double c1 = 1.0 / (2.0 * I.h1), c2 = 1.0 / (2.0 * I.h2);
  for (long long nd = (long long)blockIdx.x * blockDim.x + threadIdx.x; nd < I.nodes;
       nd += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(nd / N2), j = (int)(nd % N2);
    double s = 0.0;
    // G1 at row i' = i - 1 (central: + phi(i' + 1)) and i' = i + 1 (central: - phi(i' - 1))
    if (i - 1 > 0 && i - 1 < n1) s += c1 * l1[(long long)(i - 1) * N2 + j];
    if (i + 1 > 0 && i + 1 < n1) s -= c1 * l1[(long long)(i + 1) * N2 + j];
    if (i <= 2) s += c1 * (i == 0 ? -3.0 : (i == 1 ? 4.0 : -1.0)) * l1[j];
    if (i >= n1 - 2) s += c1 * (i == n1 ? 3.0 : (i == n1 - 1 ? -4.0 : 1.0)) * l1[(long long)n1 * N2 + j];
    const long long b = (long long)i * N2;
    if (j - 1 > 0 && j - 1 < n2) s += c2 * l2[b + j - 1];
    if (j + 1 > 0 && j + 1 < n2) s -= c2 * l2[b + j + 1];
    if (j <= 2) s += c2 * (j == 0 ? -3.0 : (j == 1 ? 4.0 : -1.0)) * l2[b];
    if (j >= n2 - 2) s += c2 * (j == n2 ? 3.0 : (j == n2 - 1 ? -4.0 : 1.0)) * l2[b + n2];
    a.lphi[I.node_off + nd] += s;
  }
}

// The interior of lambda_phi as the right-hand side of the transposed solve
// (unknown (i, j) of instance k at unk_off[k] + (i - 1) N2 + j).
__global__ void __launch_bounds__(256) k_adj_to_unknowns(DevPtrs d, AdjPtrs a) {
  const int inst = blockIdx.y;
  const Inst& I = d.inst[inst];
  for (long long nd = (long long)blockIdx.x * blockDim.x + threadIdx.x; nd < I.nodes;
       nd += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(nd / I.N2);
    if (i < 1 || i >= I.n1) continue;
    a.rhs[a.unk_off[inst] + nd - I.N2] = a.lphi[I.node_off + nd];
  }
}

// The transposed sweeps of the nested dissection (the fronts of A^T are the
// transposes of A's): forward z_S = F_SS^-T v_S, W = v_U - (F_SS^-1 F_SU)^T v_S;
// backward x_S = z_S - (F_US F_SS^-1)^T x_U.  One CTA per front, threads over
// the outputs (reading matrix rows, coalesced).
__global__ void __launch_bounds__(256) k_adj_ndT(AdjPtrs a, int f0, long long unk0, int forward) {
  extern __shared__ double s_v[];
  const NdFront F = a.nd_front[f0 + blockIdx.x];
  double* x = a.rhs + unk0;
  if (forward) {
    for (int p = threadIdx.x; p < F.s + F.u; p += blockDim.x) {
      const int2 g = *(const int2*)(a.nd_gather + F.G + 2 * p);
      double v = p < F.s ? x[a.nd_idx[F.S + p]] : 0.0;
      if (g.x >= 0) v += a.ndw[g.x];
      if (g.y >= 0) v += a.ndw[g.y];
      s_v[p] = v;
    }
    __syncthreads();
    for (int c = threadIdx.x; c < F.s + F.u; c += blockDim.x) {
      double acc = 0.0;
      if (c < F.s) {
        for (int r = 0; r < F.s; ++r) acc += a.nd_mat[F.FM + (long long)r * F.sp + c] * s_v[r];
        x[a.nd_idx[F.S + c]] = acc;
      } else {
        const int qq = c - F.s;
        for (int r = 0; r < F.s; ++r) acc += a.nd_mat[F.NB + (long long)r * F.up + qq] * s_v[r];
        a.ndw[F.W + qq] = s_v[c] - acc;
      }
    }
  } else {
    for (int p = threadIdx.x; p < F.u; p += blockDim.x) s_v[p] = x[a.nd_idx[F.U + p]];
    __syncthreads();
    for (int c = threadIdx.x; c < F.s; c += blockDim.x) {
      double acc = 0.0;
      for (int r = 0; r < F.u; ++r) acc += a.nd_mat[F.FM + (long long)(F.s + r) * F.sp + c] * s_v[r];
      x[a.nd_idx[F.S + c]] -= acc;
    }
  }
}

// After the transposed solve (lambda_b in rhs): lambda_rho = -rscale lambda_b;
// the phi_g adjoint from the Dirichlet term of the scaled right-hand side and
// from lambda_phi on the grain row; the alpha adjoint from the operator's
// derivative, -lambda_b rscale (dL/dalpha phi), and from rho's explicit
// alpha-dependence, lambda_rho rho (d ln w - dV / V).
__global__ void __launch_bounds__(256) k_adj_after_solve(DevPtrs d, AdjPtrs a, TanPtrs t, int k) {
  __shared__ double sh[256];
  const int inst = blockIdx.y;
  const Inst& I = d.inst[inst];
  const bool nofield = (I.flags & APIC_NO_FIELD) != 0;
  const double* phi = a.ck_phi + (long long)k * d.total_nodes + I.node_off;
  const double* rho = a.ck_rho + (long long)k * d.total_nodes + I.node_off;
  const double* st = t.dst + (long long)kSt * I.node_off;
  const double dl = t.dlnw[inst];
  double ga = 0.0, gp = 0.0;
  for (long long nd = (long long)blockIdx.x * blockDim.x + threadIdx.x; nd < I.nodes;
       nd += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(nd / I.N2), j = (int)(nd % I.N2);
    const long long g = I.node_off + nd;
    double lr = 0.0;
    if (i == 0) gp += a.lphi[g];
    if (i > 0 && i < I.n1 && !nofield) {
      const double lb = a.rhs[a.unk_off[inst] + nd - I.N2];
      gp += lb * t.bbc_g[g];
      double dL = 0.0;
      for (int di = -1; di <= 1; ++di)
        for (int dj = -1; dj <= 1; ++dj) {
          const int jj = j + dj;
          if (jj < 0 || jj > I.n2) continue;
          dL += st[(long long)st_slot(di, dj) * I.nodes + nd] * phi[(long long)(i + di) * I.N2 + jj];
        }
      const double sp = st[(long long)kStPole * I.nodes + nd];
      if (j == 0) dL += sp * phi[(long long)i * I.N2 + 2];
      if (j == I.n2) dL += sp * phi[(long long)i * I.N2 + I.n2 - 2];
      ga -= lb * d.rscale[g] * dL;
      lr = -d.rscale[g] * lb;
    }
    a.lrho[g] = lr;
    ga += lr * rho[nd] * (dl - t.dV[g] / d.V[g]);
  }
  const double ta = block_sum(ga, sh), tp = block_sum(gp, sh);
  if (threadIdx.x == 0) {
    if (ta != 0.0) atomicAdd(a.grad + (long long)inst * kNPar + 0, ta);
    if (tp != 0.0) atomicAdd(a.grad + (long long)inst * kNPar + 1, tp);
  }
}
#endif  // APIC_ADJOINT_COMMON

}  // namespace

template <>
void launch_adj_fwd_push<Real>(const DevPtrs& d, const AdjPtrs& a, int k, cudaStream_t s) {
  k_adj_fwd_push<<<kAdjBlocks * 4, 256, 0, s>>>(d, a, k);
}
template <>
void launch_adj_fwd_inject<Real>(const DevPtrs& d, const AdjPtrs& a, const TanPtrs& t, int k, long long max_inj,
                                 cudaStream_t s) {
  if (max_inj <= 0) return;
  const unsigned gx = (unsigned)((max_inj + 255) / 256);
  k_adj_fwd_inject<<<dim3(gx, d.n_pop), 256, 0, s>>>(d, a, t, k);
}
template <>
void launch_adj_rev_inject<Real>(const DevPtrs& d, const AdjPtrs& a, const TanPtrs& t, int k, long long max_inj,
                                 cudaStream_t s) {
  if (max_inj <= 0) return;
  const unsigned gx = (unsigned)((max_inj + 255) / 256);
  k_adj_rev_inject<<<dim3(gx, d.n_pop), 256, 0, s>>>(d, a, t, k);
}
template <>
void launch_adj_rev_push<Real>(const DevPtrs& d, const AdjPtrs& a, const TanPtrs& t, int k, cudaStream_t s) {
  k_adj_rev_push<<<kAdjBlocks, 256, 0, s>>>(d, a, t, k);
}
template <>
void launch_adj_rev_deposit<Real>(const DevPtrs& d, const AdjPtrs& a, int k, cudaStream_t s) {
  k_adj_rev_deposit<<<kAdjBlocks, 256, 0, s>>>(d, a, k);
}

#ifdef APIC_ADJOINT_COMMON
void launch_adj_values(const DevPtrs& d, const AdjPtrs& a, cudaStream_t s) {
  k_adj_values<<<(d.n_inst + 63) / 64, 64, 0, s>>>(d, a);
}
void launch_adj_surface(const DevPtrs& d, const AdjPtrs& a, const TanPtrs& t, int k, cudaStream_t s) {
  k_adj_surface<<<d.n_inst, 256, 0, s>>>(d, a, t, k);
}
void launch_adj_gradT(const DevPtrs& d, const AdjPtrs& a, cudaStream_t s) {
  k_adj_gradT<<<dim3(kRedBlocks, d.n_inst), 256, 0, s>>>(d, a);
}
void launch_adj_to_unknowns(const DevPtrs& d, const AdjPtrs& a, cudaStream_t s) {
  k_adj_to_unknowns<<<dim3(kRedBlocks, d.n_inst), 256, 0, s>>>(d, a);
}
void launch_adj_ndT(const AdjPtrs& a, int f0, int f1, long long unk0, int smem_doubles, bool forward, cudaStream_t s) {
  if (f1 <= f0) return;
  k_adj_ndT<<<f1 - f0, 256, sizeof(double) * (size_t)smem_doubles, s>>>(a, f0, unk0, forward ? 1 : 0);
}
void launch_adj_after_solve(const DevPtrs& d, const AdjPtrs& a, const TanPtrs& t, int k, cudaStream_t s) {
  k_adj_after_solve<<<dim3(kRedBlocks, d.n_inst), 256, 0, s>>>(d, a, t, k);
}
const void* adj_ndT_kernel() { return (const void*)k_adj_ndT; }
#endif

}  // namespace apic
