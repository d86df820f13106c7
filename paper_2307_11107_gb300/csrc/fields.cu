// Node-field kernels of the APIC step (arXiv:2307.11107, Sec. 2):
//   charge density from the fixed-point accumulators divided by the node
//   volumes of Eq. 5, and the right-hand side of Eqs. 6-7;
//   node gradients dphi/dx1, dphi/dx2 (used by the gather of Eq. 10);
//   surface charge and electric force on the grain (after Eq. 10);
//   per-step bookkeeping and the history of currents, forces, torque, heat flux.
#include <cuda_runtime.h>

#include "apic_internal.h"
#include "geom.cuh"

namespace apic {
namespace {

#include "fields_common.cuh"


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

// rho, the initial guess and the right-hand side at every node (rho_node),
// with per-CTA partial sums of |b|^2.
__global__ void __launch_bounds__(256) k_rho(DevPtrs d) {
  __shared__ double sh[256];
  const Inst& I = d.inst[blockIdx.y];
  double part = 0.0;
  for (long long nd = (long long)blockIdx.x * blockDim.x + threadIdx.x; nd < I.nodes;
       nd += (long long)gridDim.x * blockDim.x) {
    const double bv = rho_node(d, I, blockIdx.y, nd);
    part += bv * bv;
  }
  double tot = block_sum(part, sh);
  if (threadIdx.x == 0) d.red[((long long)blockIdx.y * kNRed + 0) * kRedBlocks + blockIdx.x] = tot;
}

// b of one instance from an externally supplied rho (Poisson-only solves).
__global__ void __launch_bounds__(256) k_b_from_rho(DevPtrs d, int inst) {
  __shared__ double sh[256];
  const Inst& I = d.inst[inst];
  double part = 0.0;
  for (long long nd = (long long)blockIdx.x * blockDim.x + threadIdx.x; nd < I.nodes;
       nd += (long long)gridDim.x * blockDim.x) {
    long long g = I.node_off + nd;
    int i = (int)(nd / I.N2);
    double bv = 0.0;
    if (i > 0 && i < I.n1) bv = -d.rho[g] * d.rscale[g] + d.bbc[g];
    d.b[g] = bv;
    part += bv * bv;
  }
  double tot = block_sum(part, sh);
  if (threadIdx.x == 0) d.red[((long long)inst * kNRed + 0) * kRedBlocks + blockIdx.x] = tot;
}

// b = the Dirichlet term of a grain at potential 1 (outer boundary at 0) and
// no charge, for the vacuum field of an isolated grain; |b|^2 partials as
// k_b_from_rho.
__global__ void __launch_bounds__(256) k_b_vacuum(DevPtrs d, int inst) {
  __shared__ double sh[256];
  const Inst& I = d.inst[inst];
  double part = 0.0;
  for (long long nd = (long long)blockIdx.x * blockDim.x + threadIdx.x; nd < I.nodes;
       nd += (long long)gridDim.x * blockDim.x) {
    long long g = I.node_off + nd;
    int i = (int)(nd / I.N2);
    double bv = i > 0 && i < I.n1 ? d.bbc_g[g] : 0.0;
    d.b[g] = bv;
    part += bv * bv;
  }
  double tot = block_sum(part, sh);
  if (threadIdx.x == 0) d.red[((long long)inst * kNRed + 0) * kRedBlocks + blockIdx.x] = tot;
}

// phi_vac = the solver's interior values, 1 on the grain row, 0 on the outer row.
__global__ void __launch_bounds__(256) k_store_vacuum(DevPtrs d, int inst) {
  const Inst& I = d.inst[inst];
  for (long long nd = (long long)blockIdx.x * blockDim.x + threadIdx.x; nd < I.nodes;
       nd += (long long)gridDim.x * blockDim.x) {
    long long g = I.node_off + nd;
    int i = (int)(nd / I.N2);
    d.phi_vac[g] = i == 0 ? 1.0 : (i == I.n1 ? 0.0 : d.phi[g]);
  }
}

// phi += dphig * phi_vac at every node of every isolated grain (the correction
// surface_block chose; the gradients are taken again afterwards).
__global__ void __launch_bounds__(256) k_float_phi(DevPtrs d) {
  const Inst& I = d.inst[blockIdx.y];
  if (!(I.flags & APIC_FLOATING)) return;
  const double dl = d.stp[blockIdx.y].dphig;
  for (long long nd = (long long)blockIdx.x * blockDim.x + threadIdx.x; nd < I.nodes;
       nd += (long long)gridDim.x * blockDim.x) {
    long long g = I.node_off + nd;
    d.phi[g] += dl * d.phi_vac[g];
  }
}

// Boltzmann electrons (APIC_BOLTZMANN): the Newton linearisation of
// L phi = -(rho_i - exp(phi)) about the current phi_k.  In the row-scaled
// system the FP64 operator's diagonal becomes diag0 - rscale exp(phi_k) and
// b = -rho_i rscale + (Dirichlet terms) + rscale exp(phi_k) (1 - phi_k); the
// |b|^2 partials as k_rho, so that the BiCGSTAB solve that follows stops at
// once when phi_k already satisfies the nonlinear equations to its
// tolerance.  The solve may also stop once its residual has fallen by eta
// (inexact Newton; eta = 0 for the last iteration).  only >= 0: that
// instance alone.
__global__ void __launch_bounds__(256) k_newton(DevPtrs d, int only, double eta) {
  __shared__ double sh[256];
  const int inst = blockIdx.y;
  const Inst& I = d.inst[inst];
  if (!(I.flags & APIC_BOLTZMANN) || (only >= 0 && inst != only)) return;
  if (blockIdx.x == 0 && threadIdx.x == 0) d.sol[inst].eta2 = eta * eta;
  double* dg = d.st64 + (long long)kSt * I.node_off + (long long)st_slot(0, 0) * I.nodes;
  double part = 0.0;
  for (long long nd = (long long)blockIdx.x * blockDim.x + threadIdx.x; nd < I.nodes;
       nd += (long long)gridDim.x * blockDim.x) {
    const long long g = I.node_off + nd;
    const int i = (int)(nd / I.N2);
    if (i == 0 || i == I.n1) continue;
    const double ph = d.phi[g], rs = d.rscale[g], rho = d.rho[g], bc = d.bbc[g], d0 = d.diag0[g];
    const double e = rs * exp(ph);
    const double bv = -rho * rs + bc + e * (1.0 - ph);
    dg[nd] = d0 - e;
    d.b[g] = bv;
    part += bv * bv;
  }
  double tot = block_sum(part, sh);
  if (threadIdx.x == 0) d.red[((long long)inst * kNRed + 0) * kRedBlocks + blockIdx.x] = tot;
}

// The linear operator's diagonal back (after a Boltzmann solve).
__global__ void __launch_bounds__(256) k_newton_end(DevPtrs d) {
  const int inst = blockIdx.y;
  const Inst& I = d.inst[inst];
  if (!(I.flags & APIC_BOLTZMANN)) return;
  double* dg = d.st64 + (long long)kSt * I.node_off + (long long)st_slot(0, 0) * I.nodes;
  for (long long nd = (long long)blockIdx.x * blockDim.x + threadIdx.x; nd < I.nodes;
       nd += (long long)gridDim.x * blockDim.x)
    dg[nd] = d.diag0[I.node_off + nd];
}

template <class Real>
struct Pair;
template <>
struct Pair<double> {
  using T = double2;
};
template <>
struct Pair<float> {
  using T = float2;
};

// Node gradients of every node (grad_node).
template <class Real>
__global__ void __launch_bounds__(256) k_gradients(DevPtrs d) {
  using R2 = typename Pair<Real>::T;
  const Inst& I = d.inst[blockIdx.y];
  for (long long nd = (long long)blockIdx.x * blockDim.x + threadIdx.x; nd < I.nodes;
       nd += (long long)gridDim.x * blockDim.x)
    grad_node<Real, R2>(d, I, nd);
}

// Surface quantities and this step's injection counts, one CTA per instance (surface_block).
__global__ void __launch_bounds__(256) k_surface(DevPtrs d) {
  __shared__ double sh[40];
  surface_block(d, blockIdx.x, sh);
}

// Close the step: injected particles become part of the population (freed
// slots reused first), the history row is written, per-step sums cleared.
__device__ void finish_injection(PopState& S, const Pop& P) {
  long long stored = S.inj_stored, nh = S.n_holes;
  if (stored <= nh) {
    S.n_holes = nh - stored;
  } else {
    long long n = S.n + (stored - nh);
    S.n = n > P.cap ? P.cap : n;
    S.n_holes = 0;
  }
  S.draws += S.n_inj;
  S.injected += S.n_inj;
  S.n_inj = 0;
  S.inj_stored = 0;
}

__global__ void k_step_end(DevPtrs d) {
  const int inst = blockIdx.x * blockDim.x + threadIdx.x;
  if (inst >= d.n_inst) return;
  const Inst& I = d.inst[inst];
  StepState& T = d.stp[inst];
  double res[2] = {0.0, 0.0};
  for (int s = 0; s < I.n_species; ++s) {
    PopState& S = d.ps[I.pop0 + s];
    finish_injection(S, d.pop[I.pop0 + s]);
    res[s] = (double)(S.loaded + S.injected - S.absorbed - S.escaped - S.dropped);
  }
  double dt = I.dt;
  step_tallies(d, inst, T.tally);
  for (int s = 0; s < I.n_species; ++s) {
    const Pop& P = d.pop[I.pop0 + s];
    unsigned long long* st = d.tfix + P.tfix_off + (long long)I.n2 * kTallyBinWords;
    for (int k = 0; k < kTallyStepWords; ++k) st[k] = 0ull;
  }
  // Boltzmann electrons reach the grain as the one-sided flux of a Maxwellian
  // of density n0 exp(phi_g) at the surface (Te = me = 1): exp(phi_g)/sqrt(2 pi)
  // per unit area and time, charge -1 each
  if (I.flags & APIC_BOLTZMANN) T.tally[0] -= exp(I.phi_g) * (1.0 / sqrt(2.0 * kPi)) * I.A_grain * dt;
  double* h = d.hist + I.hist_off + (T.step % I.hist_cap) * kNH;
  h[0] = (double)(T.step + 1) * dt;
  h[1] = T.tally[0] / dt;
  h[2] = T.tally[1] / dt;
  h[3] = T.FZ;
  h[4] = T.tally[2] / dt;
  h[5] = T.tally[3] / dt;
  h[6] = T.Q;
  h[7] = res[0];
  h[8] = res[1];
  h[9] = T.tally[4];
  h[10] = (I.flags & APIC_FLOATING) ? T.phig : I.phi_g;
  if (I.flags & APIC_FLOATING) T.qg += T.tally[0];  // charge the grain collected this step
  for (int k = 0; k < 5; ++k) T.tally[k] = 0.0;
  T.step += 1;
}

// Explicit-count surface injection outside a step: same bookkeeping.
__global__ void k_finish_injection(DevPtrs d, int pop) {
  finish_injection(d.ps[pop], d.pop[pop]);
}

}  // namespace

template <class Real>
void launch_rho(const DevPtrs& d, cudaStream_t s) {
  k_rho<<<dim3(kRedBlocks, d.n_inst), 256, 0, s>>>(d);
}
template <class Real>
void launch_gradients(const DevPtrs& d, cudaStream_t s) {
  k_gradients<Real><<<dim3(kRedBlocks, d.n_inst), 256, 0, s>>>(d);
}
template void launch_rho<double>(const DevPtrs&, cudaStream_t);
template void launch_rho<float>(const DevPtrs&, cudaStream_t);
template void launch_gradients<double>(const DevPtrs&, cudaStream_t);
template void launch_gradients<float>(const DevPtrs&, cudaStream_t);

void launch_surface(const DevPtrs& d, cudaStream_t s) { k_surface<<<d.n_inst, 256, 0, s>>>(d); }
void launch_step_end(const DevPtrs& d, cudaStream_t s) { k_step_end<<<(d.n_inst + 63) / 64, 64, 0, s>>>(d); }
void launch_finish_injection(const DevPtrs& d, int pop, cudaStream_t s) { k_finish_injection<<<1, 1, 0, s>>>(d, pop); }
void launch_b_from_rho(const DevPtrs& d, int inst, cudaStream_t s) { k_b_from_rho<<<kRedBlocks, 256, 0, s>>>(d, inst); }
void launch_b_vacuum(const DevPtrs& d, int inst, cudaStream_t s) { k_b_vacuum<<<kRedBlocks, 256, 0, s>>>(d, inst); }
void launch_store_vacuum(const DevPtrs& d, int inst, cudaStream_t s) { k_store_vacuum<<<kRedBlocks, 256, 0, s>>>(d, inst); }
void launch_float_phi(const DevPtrs& d, cudaStream_t s) { k_float_phi<<<dim3(kRedBlocks, d.n_inst), 256, 0, s>>>(d); }
void launch_newton(const DevPtrs& d, int only, double eta, cudaStream_t s) {
  k_newton<<<dim3(kRedBlocks, d.n_inst), 256, 0, s>>>(d, only, eta);
}
void launch_newton_end(const DevPtrs& d, cudaStream_t s) { k_newton_end<<<dim3(kRedBlocks, d.n_inst), 256, 0, s>>>(d); }

}  // namespace apic
