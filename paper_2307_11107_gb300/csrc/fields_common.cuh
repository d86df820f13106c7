// Per-node and per-instance bodies of the node-field work of a step (Sec. 2),
// shared by the separate kernels of fields.cu and by the prologue and
// epilogue of the block-cyclic-reduction solve (bcr.cu), so both compute the
// same values.  Included inside namespace apic::{anonymous}.
#pragma once

// rho_ij = sum_s q_s w_s (accumulated CIC weights) / V_ij (Eq. 5, as a
// product with the stored 1 / V_ij: FP64 division is slow on this GPU); the
// accumulators are cleared for the next deposit; the initial guess of this
// step's solve (previous phi, or its linear extrapolation); the right-hand
// side b = rscale * (-rho) + (Dirichlet terms; an isolated grain, APIC_FLOATING,
// at its last potential phig).  Returns b at the node.
// Every load comes before the first store: a load placed after a store that
// might alias it waits for that store, which made this node loop a chain of
// memory round trips.
__device__ __forceinline__ double rho_node(const DevPtrs& d, const Inst& I, int inst, long long nd) {
  const long long g = I.node_off + nd;
  const int ns = I.n_species;  // 1 or 2
  const int i = (int)(nd / I.N2);
  const bool interior = i > 0 && i < I.n1;
  const bool extrap = I.guess && d.stp[inst].step >= 2;
  const Pop& P0 = d.pop[I.pop0];
  const Pop& P1 = d.pop[I.pop0 + (ns > 1 ? 1 : 0)];
  const long long o0 = P0.acc_off + nd, o1 = P1.acc_off + nd;
  const double s0 = P0.dep_scale, s1 = P1.dep_scale;
  const unsigned long long a0 = d.acc[o0];
  const unsigned long long a1 = ns > 1 ? d.acc[o1] : 0ull;
  const double vinv = d.Vinv[g];
  const bool fl = (I.flags & APIC_FLOATING) != 0;
  double ph = 0.0, prev = 0.0, rs = 0.0, bc = 0.0, bg = 0.0, dg = 0.0;
  if (interior) {
    ph = d.phi[g];
    prev = d.phi_prev[g];
    rs = d.rscale[g];
    bc = d.bbc[g];
    if (fl) {
      bg = d.bbc_g[g];
      dg = d.stp[inst].phig - I.phi_g;
    }
  }
  double q = 0.0;
  q += s0 * (double)a0;
  if (ns > 1) q += s1 * (double)a1;
  const double rho = q * vinv;
  const double bv = interior ? -rho * rs + (fl ? bc + dg * bg : bc) : 0.0;
  d.acc[o0] = 0ull;
  if (ns > 1) d.acc[o1] = 0ull;
  d.rho[g] = rho;
  if (interior) {
    if (extrap) d.phi[g] = 2.0 * ph - prev;
    d.phi_prev[g] = ph;
  }
  d.b[g] = bv;
  return bv;
}

// Node gradients: central differences inside, one-sided second order on the
// four edges (Sec. 2: derivatives of phi taken numerically at the nodes),
// scaled by the stored 1 / (2 h).
template <class Real, class R2>
__device__ __forceinline__ void grad_node(const DevPtrs& d, const Inst& I, long long nd) {
  const double* p = d.phi + I.node_off;
  const bool nofield = (I.flags & APIC_NO_FIELD) != 0;
  const int n1 = I.n1, n2 = I.n2, N2 = I.N2;
  const int i = (int)(nd / N2), j = (int)(nd % N2);
  double g1 = 0.0, g2 = 0.0;
  if (!nofield) {
    if (i == 0) g1 = (-3.0 * p[j] + 4.0 * p[N2 + j] - p[2 * N2 + j]) * I.i2h1;
    else if (i == n1) g1 = (3.0 * p[n1 * N2 + j] - 4.0 * p[(n1 - 1) * N2 + j] + p[(n1 - 2) * N2 + j]) * I.i2h1;
    else g1 = (p[(i + 1) * N2 + j] - p[(i - 1) * N2 + j]) * I.i2h1;
    const long long b = (long long)i * N2;
    if (j == 0) g2 = (-3.0 * p[b] + 4.0 * p[b + 1] - p[b + 2]) * I.i2h2;
    else if (j == n2) g2 = (3.0 * p[b + n2] - 4.0 * p[b + n2 - 1] + p[b + n2 - 2]) * I.i2h2;
    else g2 = (p[b + j + 1] - p[b + j - 1]) * I.i2h2;
  }
  R2 v;
  v.x = (Real)g1;
  v.y = (Real)g2;
  ((R2*)d.G)[I.node_off + nd] = v;
  if constexpr (sizeof(Real) == sizeof(float)) {
    if (d.H) {  // the pair table: this node's half of its own entry and of its left neighbour's
      float2* H2 = (float2*)d.H;
      const float2 w = make_float2((float)v.x, (float)v.y);
      H2[2 * (I.node_off + nd)] = w;
      if (j > 0) H2[2 * (I.node_off + nd) - 1] = w;
    }
  }
}

// Fixed-order block sum (warp shuffles, then warp 0 over the warp sums); any
// blockDim that is a multiple of 32, at most 1024; sh holds 33 doubles.
__device__ __forceinline__ double block_total(double v, double* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (int)(blockDim.x >> 5);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  if (warp == 0) {
    double t = lane < nw ? sh[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if (lane == 0) sh[32] = t;
  }
  __syncthreads();
  const double r = sh[32];
  __syncthreads();
  return r;
}

// Surface charge sigma = E_n = -(dphi/dx1)|grad x1| on x1 = -1, grain charge
// Q = int sigma dA and electric force F_Z = int (sigma^2/2) n_Z dA with dA of
// Eq. 4 (trapezoid over the x2 nodes, geometry tabulated at set-up).  Thread
// 0 also draws this step's injection count from the fractional carry.  One
// CTA per instance.
//
// Isolated grain (APIC_FLOATING): the problem is linear, so adding
// dphig * phi_vac (the vacuum field of a grain at 1, outer boundary at 0)
// moves the grain to phig + dphig and its charge to Q + dphig * C_vac, C_vac
// the charge of phi_vac.  dphig is chosen so that the charge is the one the
// grain holds (fixed at the first step, then grown by what it absorbs); E_n
// and F_Z here are those of the corrected field, whose nodes the next kernel
// (k_float_phi) updates.
__device__ __forceinline__ void surface_block(const DevPtrs& d, int inst, double* sh) {
  const Inst& I = d.inst[inst];
  const bool nofield = (I.flags & APIC_NO_FIELD) != 0;
  const bool fl = (I.flags & APIC_FLOATING) != 0;
  double q = 0.0, fz = 0.0, cv = 0.0;
  const double* p = d.phi + I.node_off;
  const double* pv = d.phi_vac + I.node_off;
  const int N2 = I.N2;
  const double* geo = d.sgeo + 4 * I.en_off;  // |grad x1|, n_Z, dA/dx2, trapezoid weight per node
  for (int j = threadIdx.x; j <= I.n2; j += blockDim.x) {
    double En = 0.0;
    if (!nofield) {
      double g = geo[4 * j + 0], nZ = geo[4 * j + 1], dA = geo[4 * j + 2], tw = geo[4 * j + 3];
      double G1 = (-3.0 * p[j] + 4.0 * p[N2 + j] - p[2 * N2 + j]) / (2.0 * I.h1);
      En = -G1 * g;
      q += tw * En * dA;
      fz += tw * 0.5 * En * En * nZ * dA;
      if (fl) cv += tw * (-(-3.0 * pv[j] + 4.0 * pv[N2 + j] - pv[2 * N2 + j]) / (2.0 * I.h1) * g) * dA;
    }
    d.en[I.en_off + j] = En;
  }
  double Q = block_total(q, sh);
  double FZ = block_total(fz, sh);
  if (fl) {
    StepState& T = d.stp[inst];
    const double CV = block_total(cv, sh);
    const double qg = T.qg_set != 0.0 ? T.qg : Q;
    const double dl = (qg - Q) / CV;
    __syncthreads();  // every thread has read T before thread 0 writes it
    fz = 0.0;
    for (int j = threadIdx.x; j <= I.n2; j += blockDim.x) {
      double g = geo[4 * j + 0], nZ = geo[4 * j + 1], dA = geo[4 * j + 2], tw = geo[4 * j + 3];
      double Ev = -(-3.0 * pv[j] + 4.0 * pv[N2 + j] - pv[2 * N2 + j]) / (2.0 * I.h1) * g;
      double En = d.en[I.en_off + j] + dl * Ev;
      fz += tw * 0.5 * En * En * nZ * dA;
      d.en[I.en_off + j] = En;
    }
    FZ = block_total(fz, sh);
    Q += dl * CV;
    if (threadIdx.x == 0) {
      T.qg = qg;
      T.qg_set = 1.0;
      T.dphig = dl;
      T.phig += dl;
    }
  }
  if (threadIdx.x == 0) {
    d.stp[inst].Q = Q;
    d.stp[inst].FZ = FZ;
    if (!(Q == Q) || !(FZ == FZ) || Q - Q != 0.0) atomicOr(d.err, kErrNonFinite);
    for (int s = 0; s < I.n_species; ++s) {
      PopState& S = d.ps[I.pop0 + s];
      const Pop& P = d.pop[I.pop0 + s];
      if (I.flags & APIC_NO_INJECT) {
        S.n_inj = 0;
      } else {
        double c = S.carry + P.lam;
        double nk = floor(c);
        S.carry = c - nk;
        S.n_inj = (long long)nk;
      }
      S.inj_stored = 0;
    }
  }
}
