// pibm_fluid_sums_noalloc: total mass and fluid momentum of populations that the
// caller holds on the device, computed without any device allocation.
//
// It is the fixed-order reduction behind pibm_invariants, reading plain FP64
// populations in the ABI layout instead of a handle's stored state, with its
// partial sums in a file-scope static device array instead of a workspace.
// That array (NA_SLOTS x NA_MAX_PARTIALS doubles, 128 KiB) exists on every GPU
// that loads the library, for the life of the process.
#include <mutex>

#include "pibm_internal.cuh"

namespace {

constexpr int NA_THREADS = 256;
constexpr int NA_CHUNK = 4096;           // cells summed by one CTA
constexpr int NA_MAX_PARTIALS = 4096;    // CTAs per call, one partial each
constexpr long long NA_MAX_CELLS = (long long)NA_CHUNK * NA_MAX_PARTIALS;  // 16,777,216
constexpr int NA_SLOTS = 4;              // rho, jx, jy, jz
constexpr int NA_MAX_DEVICES = 64;

// Partial sums [NA_SLOTS][NA_MAX_PARTIALS]. Every call overwrites the partials it
// uses before reading them, so nothing has to start at zero.
static __device__ __align__(256) double na_scratch[NA_SLOTS * NA_MAX_PARTIALS];

template <int NV>
__device__ void na_block_tree(double (&v)[NV], double* sm) {
#pragma unroll
  for (int k = 0; k < NV; ++k) sm[k * NA_THREADS + threadIdx.x] = v[k];
  __syncthreads();
  for (int s = NA_THREADS / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) {
#pragma unroll
      for (int k = 0; k < NV; ++k)
        sm[k * NA_THREADS + threadIdx.x] += sm[k * NA_THREADS + threadIdx.x + s];
    }
    __syncthreads();
  }
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = sm[k * NA_THREADS];
}

// CTA b sums the cells [b * NA_CHUNK, (b + 1) * NA_CHUNK): each thread a fixed
// strided subset, then a fixed tree, so the result does not depend on timing.
template <int Q>
__global__ void __launch_bounds__(NA_THREADS) k_na_partials(const double* __restrict__ f,
                                                            long long ncell,
                                                            double* __restrict__ part) {
  using L = pibm::Lattice<Q>;
  constexpr int D = L::D;
  __shared__ double sm[(D + 1) * NA_THREADS];
  double acc[D + 1];
#pragma unroll
  for (int k = 0; k <= D; ++k) acc[k] = 0.0;
  const long long c0 = (long long)blockIdx.x * NA_CHUNK;
  const long long c1 = c0 + NA_CHUNK < ncell ? c0 + NA_CHUNK : ncell;
  for (long long c = c0 + threadIdx.x; c < c1; c += NA_THREADS) {
#pragma unroll
    for (int a = 0; a < Q; ++a) {
      const double v = f[(long long)a * ncell + c];
      acc[0] += v;
#pragma unroll
      for (int k = 0; k < D; ++k)
        if (L::e(a, k)) acc[k + 1] += L::e(a, k) * v;
    }
  }
  na_block_tree<D + 1>(acc, sm);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k <= D; ++k) part[k * NA_MAX_PARTIALS + blockIdx.x] = acc[k];
  }
}

template <int NV>
__global__ void __launch_bounds__(NA_THREADS) k_na_final(const double* __restrict__ part, int nb,
                                                         double* __restrict__ out) {
  __shared__ double sm[NV * NA_THREADS];
  double acc[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) acc[k] = 0.0;
  for (int b = threadIdx.x; b < nb; b += NA_THREADS) {
#pragma unroll
    for (int k = 0; k < NV; ++k) acc[k] += part[k * NA_MAX_PARTIALS + b];
  }
  na_block_tree<NV>(acc, sm);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) out[k] = acc[k];
  }
}

std::mutex g_na_mu;
double* g_na_ptr[NA_MAX_DEVICES] = {};

// Device address of na_scratch on the current device. In host code the name
// na_scratch is only a host-side stand-in, so the address is looked up once per
// device with that device current and cached.
int scratch_for_current_device(double** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) {
    pibm::record_cuda_error("cudaGetDevice", e != cudaSuccess ? e : cudaErrorInvalidDevice);
    cudaGetLastError();
    return PIBM_ECUDA;
  }
  std::lock_guard<std::mutex> lock(g_na_mu);
  if (!g_na_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, na_scratch);
    if (e != cudaSuccess || !p) {
      pibm::record_cuda_error("cudaGetSymbolAddress", e != cudaSuccess ? e : cudaErrorInvalidSymbol);
      cudaGetLastError();
      return PIBM_ECUDA;
    }
    g_na_ptr[dev] = (double*)p;
  }
  *out = g_na_ptr[dev];
  return PIBM_OK;
}

}  // namespace

extern "C" int pibm_fluid_sums_noalloc(const double* f, int lattice, const int64_t n[3],
                                       double* out, void* stream) {
  if (!f || !out || !n) return PIBM_EINVAL;
  if (lattice != PIBM_D2Q9 && lattice != PIBM_D3Q15 && lattice != PIBM_D3Q19) return PIBM_EINVAL;
  if (n[0] < 1 || n[1] < 1 || n[2] < 1) return PIBM_EINVAL;
  if (lattice == PIBM_D2Q9 && n[2] != 1) return PIBM_EINVAL;
  long long ncell = 1;
  for (int k = 0; k < 3; ++k) {
    // checked before multiplying, so the product never overflows
    if (n[k] > NA_MAX_CELLS / ncell) return PIBM_ETOOBIG;  // beyond the static scratch
    ncell *= n[k];
  }
  // an error left pending by an earlier, unrelated call on this thread is
  // cleared here, so that it is not reported as this call's launch failure
  cudaGetLastError();
  double* part = nullptr;
  int rc = scratch_for_current_device(&part);
  if (rc != PIBM_OK) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const int nb = (int)((ncell + NA_CHUNK - 1) / NA_CHUNK);
  switch (lattice) {
    case PIBM_D2Q9:
      k_na_partials<9><<<nb, NA_THREADS, 0, st>>>(f, ncell, part);
      k_na_final<3><<<1, NA_THREADS, 0, st>>>(part, nb, out);
      break;
    case PIBM_D3Q15:
      k_na_partials<15><<<nb, NA_THREADS, 0, st>>>(f, ncell, part);
      k_na_final<4><<<1, NA_THREADS, 0, st>>>(part, nb, out);
      break;
    default:
      k_na_partials<19><<<nb, NA_THREADS, 0, st>>>(f, ncell, part);
      k_na_final<4><<<1, NA_THREADS, 0, st>>>(part, nb, out);
      break;
  }
  const cudaError_t le = cudaGetLastError();
  if (le != cudaSuccess) {
    pibm::record_cuda_error("pibm_fluid_sums_noalloc launch", le);
    return PIBM_ECUDA;
  }
  return PIBM_OK;
}
