// jz_static.cu -- diagnostics of a state held in the caller's device arrays,
// computed without any device memory beyond the caller's inputs and output.
//
// Who needs this: code that can only work with device arrays it was handed
// and must not obtain more device memory -- for example a plug-in that a host
// framework calls with its input and output buffers, or a serving process
// that reserved all of its device memory at start-up and treats any later
// allocation as a failure.  Such callers cannot size and pass the scratch
// area that jz_diagnostics takes from a grid's buffer, so this entry point
// keeps its reduction scratch in a fixed, file-scope device array instead.
//
// The scratch array is shared by every call in the process on a device and
// keeps the contents of the last call; two calls whose kernels overlap on the
// GPU (different streams, no ordering between them) race on it.  Calls on one
// stream, or otherwise ordered, are safe.
#include <cmath>

#include "jz_internal.h"

namespace jz {

namespace {

constexpr int SD_THREADS = 256;
constexpr long long SD_CHUNK = 65536;  // nodes reduced by one block
constexpr int SD_MAX_CHUNKS = 4096;    // blocks the scratch can hold
constexpr int SD_WORDS = 11;           // same per-block record as the grid diagnostics
constexpr long long SD_MAX_NODES = SD_CHUNK * SD_MAX_CHUNKS;  // 268,435,456

// per-block partial records, then one word for the last-block counter
// (4096 x 11 x 8 bytes + 256 bytes, about 352 KB per device)
static __device__ __align__(256) double sd_scratch[SD_MAX_CHUNKS * SD_WORDS + 32];

template <typename ST>
__global__ void __launch_bounds__(SD_THREADS) k_diag_static(long long n, const ST* __restrict__ Q,
                                                            const double* __restrict__ vol, double gamma,
                                                            double* scratch, double* out) {
  double* partial = scratch;
  unsigned int* counter = reinterpret_cast<unsigned int*>(scratch + SD_MAX_CHUNKS * SD_WORDS);
  const ST gm1s = (ST)(gamma - 1.0), gs = (ST)gamma;
  double acc[SD_WORDS] = {0, 0, 0, 0, 0, INFINITY, -INFINITY, INFINITY, -INFINITY, 0, 0};
  const long long lo = (long long)blockIdx.x * SD_CHUNK;
  const long long hi = lo + SD_CHUNK < n ? lo + SD_CHUNK : n;
  for (long long t = lo + threadIdx.x; t < hi; t += SD_THREADS) {
    double q[5];
    bool finite = true;
    for (int v = 0; v < 5; ++v) {
      q[v] = (double)Q[(long long)v * n + t];
      finite = finite && isfinite(q[v]);
    }
    if (!finite) { acc[10] += 1.0; continue; }
    const double V = vol[t];
    for (int v = 0; v < 5; ++v) acc[v] += q[v] * V;
    // pressure and squared Mach number in the state's type, as the grid
    // diagnostics compute them
    ST qs[5], p, m2;
    for (int v = 0; v < 5; ++v) qs[v] = Q[(long long)v * n + t];
    diag_node<ST>(qs, gm1s, gs, p, m2);
    acc[5] = fmin(acc[5], q[0]);
    acc[6] = fmax(acc[6], q[0]);
    acc[7] = fmin(acc[7], (double)p);
    acc[8] = fmax(acc[8], (double)p);
    acc[9] = fmax(acc[9], (double)m2);
  }
  __shared__ double sh[SD_WORDS][SD_THREADS];
  for (int c = 0; c < SD_WORDS; ++c) sh[c][threadIdx.x] = acc[c];
  __syncthreads();
  for (int half = SD_THREADS / 2; half > 0; half >>= 1) {  // fixed-order tree
    if ((int)threadIdx.x < half) {
      const int o = threadIdx.x + half;
      for (int c = 0; c < 5; ++c) sh[c][threadIdx.x] += sh[c][o];
      sh[5][threadIdx.x] = fmin(sh[5][threadIdx.x], sh[5][o]);
      sh[6][threadIdx.x] = fmax(sh[6][threadIdx.x], sh[6][o]);
      sh[7][threadIdx.x] = fmin(sh[7][threadIdx.x], sh[7][o]);
      sh[8][threadIdx.x] = fmax(sh[8][threadIdx.x], sh[8][o]);
      sh[9][threadIdx.x] = fmax(sh[9][threadIdx.x], sh[9][o]);
      sh[10][threadIdx.x] += sh[10][o];
    }
    __syncthreads();
  }
  __shared__ bool last;
  if (threadIdx.x == 0) {
    for (int c = 0; c < SD_WORDS; ++c) partial[(long long)blockIdx.x * SD_WORDS + c] = sh[c][0];
    __threadfence();
    last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {  // the last block combines the records in block order
    __threadfence();
    const volatile double* P = partial;
    double r[SD_WORDS] = {0, 0, 0, 0, 0, INFINITY, -INFINITY, INFINITY, -INFINITY, 0, 0};
    for (int b = 0; b < (int)gridDim.x; ++b) {
      const volatile double* x = P + (long long)b * SD_WORDS;
      for (int c = 0; c < 5; ++c) r[c] += x[c];
      r[5] = fmin(r[5], x[5]);
      r[6] = fmax(r[6], x[6]);
      r[7] = fmin(r[7], x[7]);
      r[8] = fmax(r[8], x[8]);
      r[9] = fmax(r[9], x[9]);
      r[10] += x[10];
    }
    for (int c = 0; c < SD_WORDS; ++c) out[c] = r[c];
    out[9] = sqrt(r[9]);  // maximum Mach number
  }
}

int static_fail(int code, const char* msg) { return record_error(code, msg); }

}  // namespace

}  // namespace jz

using namespace jz;

extern "C" int jz_state_diagnostics_static(long long n_nodes, int fp64, const void* Q, const double* vol,
                                           double gamma, double* out, void* stream) {
  if (n_nodes < 0) return static_fail(JZ_EINVAL, "negative node count");
  if (n_nodes > SD_MAX_NODES) return static_fail(JZ_EINVAL, "node count exceeds the static-scratch maximum 268435456");
  if (!Q || !vol || !out) return static_fail(JZ_EINVAL, "null device pointer");
  if (fp64 != 0 && fp64 != 1) return static_fail(JZ_EINVAL, "fp64 must be 0 or 1");
  if (!(gamma > 1.0)) return static_fail(JZ_EINVAL, "gamma must exceed 1");
  // The host-side name of the static array is not a device address.  Look
  // the address up on every call, for the device (and context) current now:
  // the lookup allocates nothing, and a cached address would go stale once
  // the device is reset and the library's device code loaded again.  The
  // first call on a device also loads that device code (lazy loading).
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, sd_scratch);
  if (e != cudaSuccess || !p) return static_fail(JZ_ECUDA, "cudaGetSymbolAddress of the static scratch failed");
  double* scratch = (double*)p;
  cudaStream_t s = (cudaStream_t)stream;
  // The last-block counter must start at zero.  This memset, enqueued ahead
  // of the kernel on the same stream, is what guarantees it; it also clears
  // a count left by an earlier call that did not complete.
  if (cudaMemsetAsync(scratch + SD_MAX_CHUNKS * SD_WORDS, 0, sizeof(unsigned int), s) != cudaSuccess)
    return static_fail(JZ_ECUDA, "clearing the static counter failed");
  const long long blocks_ll = n_nodes > 0 ? (n_nodes + SD_CHUNK - 1) / SD_CHUNK : 1;
  const int blocks = (int)blocks_ll;
  if (fp64)
    k_diag_static<double><<<blocks, SD_THREADS, 0, s>>>(n_nodes, (const double*)Q, vol, gamma, scratch, out);
  else
    k_diag_static<float><<<blocks, SD_THREADS, 0, s>>>(n_nodes, (const float*)Q, vol, gamma, scratch, out);
  count_launches(1);
  e = cudaGetLastError();
  if (e != cudaSuccess) return static_fail(JZ_ECUDA, cudaGetErrorString(e));
  return JZ_OK;
}
