// apic_deposit_static: the cloud-in-cell charge deposit with its 64-bit
// fixed-point accumulator in library-owned static device memory, for callers
// that cannot allocate device memory themselves.
//
// Some callers cannot call cudaMalloc where they need a density: a component
// that runs under a device-memory budget owned by another part of the
// program, a host framework that only hands out the buffers it manages, or a
// latency-critical loop that must not enter the allocator.  This entry point
// takes the caller's particle positions, node volumes and output array and
// needs no other device memory: its scratch is the file-scope array below,
// which every GPU that loads the library keeps until the process exits
// (8 MiB per device).  The first call on a device looks up the array's device
// address; make that first call before any stream capture.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "../../include/apic.h"

namespace {

constexpr long long kStaticNodes = 1ll << 20;  // node capacity of the static accumulator
constexpr int kMaxDevices = 64;

// Shared by every call on a device: calls that overlap on the GPU race on it.
__device__ __align__(256) unsigned long long g_static_acc[kStaticNodes];

std::mutex g_mu;
void* g_acc_ptr[kMaxDevices] = {};

// Device address of the static accumulator on the current device, looked up
// once per device (host code cannot use the symbol's name as an address).
cudaError_t static_acc(unsigned long long** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_acc_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_acc);
    if (e != cudaSuccess) return e;
    g_acc_ptr[dev] = p;
  }
  *out = (unsigned long long*)g_acc_ptr[dev];
  return cudaSuccess;
}

__global__ void k_clear(unsigned long long* acc, long long nodes) {
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < nodes;
       k += (long long)gridDim.x * blockDim.x)
    acc[k] = 0ull;
}

// Bilinear (cloud-in-cell) weights of each particle in the logical (x1, x2)
// grid, rounded to F fractional bits and added with 64-bit integer atomics
// (order-independent sums).  A particle outside [-1, x1_outer] x [-1, 1], or
// with a non-finite coordinate, carries no charge onto the grid (as a freed
// or escaped slot of a simulation does) and is skipped.
__global__ void k_weigh(unsigned long long* acc, const double* x1, const double* x2, long long n, int n1, int n2,
                        double x1_outer, double h1, double h2, int F) {
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x) {
    const double a = x1[k], c = x2[k];
    if (!(a >= -1.0 && a <= x1_outer && c >= -1.0 && c <= 1.0)) continue;  // NaN fails too
    double u1 = (a + 1.0) / h1, u2 = (c + 1.0) / h2;
    int i = (int)floor(u1), j = (int)floor(u2);
    i = i < 0 ? 0 : (i > n1 - 1 ? n1 - 1 : i);
    j = j < 0 ? 0 : (j > n2 - 1 ? n2 - 1 : j);
    double f1 = u1 - i, f2 = u2 - j;
    f1 = f1 < 0.0 ? 0.0 : (f1 > 1.0 ? 1.0 : f1);
    f2 = f2 < 0.0 ? 0.0 : (f2 > 1.0 ? 1.0 : f2);
    double sc = ldexp(1.0, F), g1 = 1.0 - f1, g2 = 1.0 - f2;
    long long N2 = n2 + 1, b = (long long)i * N2 + j;
    atomicAdd(acc + b, (unsigned long long)__double2ll_rn(g1 * g2 * sc));
    atomicAdd(acc + b + N2, (unsigned long long)__double2ll_rn(f1 * g2 * sc));
    atomicAdd(acc + b + 1, (unsigned long long)__double2ll_rn(g1 * f2 * sc));
    atomicAdd(acc + b + N2 + 1, (unsigned long long)__double2ll_rn(f1 * f2 * sc));
  }
}

__global__ void k_density(const unsigned long long* acc, const double* V, double* rho, long long nodes, double scale) {
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < nodes;
       k += (long long)gridDim.x * blockDim.x)
    rho[k] = scale * (double)acc[k] / V[k];
}

}  // namespace

extern "C" int apic_deposit_static(const apic_grid_t* grid, const double* x1, const double* x2, int64_t n,
                                   double qw, const double* volume, double* rho, void* stream) {
  if (!grid || !volume || !rho || n < 0 || (n > 0 && (!x1 || !x2))) return APIC_ERR_INVALID_ARG;
  if (grid->n1 < 1 || grid->n2 < 1 || !(grid->x1_outer > -1.0 && grid->x1_outer < 0.0)) return APIC_ERR_INVALID_ARG;
  long long nodes = (long long)(grid->n1 + 1) * (grid->n2 + 1);
  if (nodes > kStaticNodes) return APIC_ERR_INVALID_ARG;  // larger than the static scratch
  if (n >= (1ll << 40)) return APIC_ERR_INVALID_ARG;
  unsigned long long* acc = nullptr;
  if (static_acc(&acc) != cudaSuccess) return APIC_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  int bits = 0;
  for (long long v = n; v > 0; v >>= 1) ++bits;
  int F = 62 - bits;  // n weights of at most 2^F each cannot overflow 2^62
  int gb = (int)((nodes + 255) / 256);
  gb = gb > 4096 ? 4096 : gb;
  k_clear<<<gb, 256, 0, s>>>(acc, nodes);
  if (cudaGetLastError() != cudaSuccess) return APIC_ERR_CUDA;
  if (n > 0) {
    double h1 = (grid->x1_outer + 1.0) / grid->n1, h2 = 2.0 / grid->n2;
    long long wb = (n + 255) / 256;
    wb = wb > 16384 ? 16384 : wb;  // grid-stride loop beyond 2^22 particles
    k_weigh<<<(unsigned)wb, 256, 0, s>>>(acc, x1, x2, n, grid->n1, grid->n2, grid->x1_outer, h1, h2, F);
    if (cudaGetLastError() != cudaSuccess) return APIC_ERR_CUDA;  // rho is not written
  }
  k_density<<<gb, 256, 0, s>>>(acc, volume, rho, nodes, qw * ldexp(1.0, -F));
  return cudaGetLastError() == cudaSuccess ? APIC_OK : APIC_ERR_CUDA;
}
