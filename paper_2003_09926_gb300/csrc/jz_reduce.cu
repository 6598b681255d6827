// jz_reduce.cu -- per-step time-step reduction and on-demand diagnostics.
//
// Both kernels run on a fixed grid of RED_THREADS-thread blocks: each
// thread visits grid nodes in a fixed grid-stride order, blocks reduce with
// a fixed shuffle/shared-memory tree, and the last block to finish combines
// the per-block partials in block order.  Results are therefore bitwise
// reproducible run to run (no floating-point atomics).
//
// Time step (reading of the paper: the validation run uses a fixed dt,
// Section 6; the CFL form is this build's): dt = CFL / max over grid nodes of
//   sum_k J (|S^k . u| + c |S^k|) + 2 nu_max J^2 sum_k |S^k|^2,
//   nu_max = max(4/3, gamma/Pr) mu(T) / rho.
#include <cmath>

#include "jz_internal.h"

namespace jz {

namespace {

// Grids of the two reductions: one resident wave each at 256 threads (the
// FP32 diagnostics kernel holds three blocks per SM, the time-step kernel
// two), so every block streams one equal share of the rows; more blocks than
// fit leave the last wave partly idle (diagnostics of the 256x192x192 FP32
// grid: 0.086 ms with 456 blocks, 0.110 ms with 1216).  Both fit the
// RED_BLOCKS partials.
int red_grid(int per_sm) {
  const int b = per_sm * device_sm_count();
  return b < RED_BLOCKS ? b : RED_BLOCKS;
}

template <typename T>
__device__ __forceinline__ T sutherland(T mu_inf, T s1, T temp) {
  return mu_inf * temp * sqrt(temp) * (T(1) + s1) / (temp + s1);
}

__device__ __forceinline__ double warp_max(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Returns true in exactly one thread of the last block to finish.
__device__ bool last_block(unsigned int* counter) {
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned int prev = atomicAdd(counter, 1u);
    last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  return last;
}


// Diagnostics records: [0..4] sum Q_v/J, [5] rho min, [6] rho max, [7] p min,
// [8] p max, [9] max of the squared Mach number, [10] non-finite count.
// Combine record o into record r.
__device__ __forceinline__ void diag_combine(double* r, const volatile double* o) {
  for (int c = 0; c < 5; ++c) r[c] += o[c];
  r[5] = fmin(r[5], o[5]);
  r[6] = fmax(r[6], o[6]);
  r[7] = fmin(r[7], o[7]);
  r[8] = fmax(r[8], o[8]);
  r[9] = fmax(r[9], o[9]);
  r[10] += o[10];
}

// The records of a block's threads (acc) reduced by a fixed tree into
// sh[.][0]; ends with a barrier.
__device__ __forceinline__ void diag_block_tree(const double* acc, double (*sh)[RED_THREADS]) {
  for (int c = 0; c < DIAG_WORDS; ++c) sh[c][threadIdx.x] = acc[c];
  __syncthreads();
  for (int half = RED_THREADS / 2; half > 0; half >>= 1) {
    if ((int)threadIdx.x < half) {
      double r[DIAG_WORDS], o[DIAG_WORDS];
      for (int c = 0; c < DIAG_WORDS; ++c) {
        r[c] = sh[c][threadIdx.x];
        o[c] = sh[c][threadIdx.x + half];
      }
      diag_combine(r, o);
      for (int c = 0; c < DIAG_WORDS; ++c) sh[c][threadIdx.x] = r[c];
    }
    __syncthreads();
  }
}

// Last block: combine the nb block records (in block order per thread, then
// the fixed tree: the same order whichever block is last) and publish the
// diagnostics of the state in the grid's device record.
__device__ __forceinline__ void diag_finish(const double* partial, int nb, Scalars* sc, double (*sh)[RED_THREADS]) {
  const volatile double* P = partial;
  double r[DIAG_WORDS] = {0, 0, 0, 0, 0, INFINITY, -INFINITY, INFINITY, -INFINITY, 0, 0};
  for (int b = threadIdx.x; b < nb; b += blockDim.x) diag_combine(r, P + (long long)b * DIAG_WORDS);
  __syncthreads();
  diag_block_tree(r, sh);
  if (threadIdx.x == 0) {
    for (int c = 0; c < DIAG_WORDS; ++c) sc->diag[c] = sh[c][0];
    sc->diag[9] = sqrt(sh[9][0]);  // maximum Mach number
    jz_diag& o = sc->out;
    o.time = sc->time;
    o.step = sc->step;
    o.dt = sc->dt;
    for (int v = 0; v < 5; ++v) o.sum[v] = sc->diag[v];
    o.rho_min = sc->diag[5];
    o.rho_max = sc->diag[6];
    o.p_min = sc->diag[7];
    o.p_max = sc->diag[8];
    o.mach_max = sc->diag[9];
    o.nonfinite = (int64_t)sc->diag[10];
  }
}

// Per-thread diagnostics accumulator of one state type.
template <typename ST>
struct DiagAcc {
  RunSum<ST> sum[5];
  ST rmin = ST(INFINITY), rmax = ST(-INFINITY), pmin = ST(INFINITY), pmax = ST(-INFINITY), m2max = ST(0);
  double nonfinite = 0.0;
  __device__ __forceinline__ void node(const ST q[5], ST Jn, ST gm1, ST g) {
    bool finite = true;
#pragma unroll
    for (int v = 0; v < 5; ++v) finite = finite && isfinite(q[v]);
    if (!finite) {
      nonfinite += 1.0;
      return;
    }
    const ST vol = ST(1) / Jn;
#pragma unroll
    for (int v = 0; v < 5; ++v) sum[v].add(q[v] * vol);
    ST p, m2;
    diag_node<ST>(q, gm1, g, p, m2);
    const ST rho = q[0];
    rmin = rho < rmin ? rho : rmin;
    rmax = rho > rmax ? rho : rmax;
    pmin = p < pmin ? p : pmin;
    pmax = p > pmax ? p : pmax;
    m2max = m2 > m2max ? m2 : m2max;
  }
  __device__ __forceinline__ void record(double* acc) const {
    for (int v = 0; v < 5; ++v) acc[v] = sum[v].value();
    acc[5] = (double)rmin;
    acc[6] = (double)rmax;
    acc[7] = (double)pmin;
    acc[8] = (double)pmax;
    acc[9] = (double)m2max;
    acc[10] = nonfinite;
  }
};

// DIAG: every block also forms the diagnostics of the state it reads (its
// record after the RED_BLOCKS rate partials) and the last block publishes
// them, as k_diag does.
template <typename ST, typename MT, bool DIAG = false>
__device__ __forceinline__ void timestep_body(const Layout& L, const FlowC& F, const ST* __restrict__ Q,
                                              const MT* __restrict__ M, Scalars* sc, double* partial, double cfl,
                                              bool finalize = true) {
  const ST g = flow_const<ST>(F.gamma, F.gamma_f), gm1 = flow_const<ST>(F.gm1, F.gm1_f);
  const ST mu_inf = (ST)F.mu_inf, s1 = (ST)F.s1;
  const ST vfac = flow_const<ST>(F.vfac, F.vfac_f);
  // the maximum is taken in the arithmetic type: exact, and the same value
  // as a maximum of the widened rates
  ST best_s = ST(0);
  DiagAcc<ST> dg;
  // the nodes are taken as items of 32 consecutive i (item = ch + nch (j +
  // nj k), ch the chunk of i); warp w of the fixed grid takes items 4w ..
  // 4w + 3, then the next four after all warps, one node per lane and item,
  // with the loads of all four issued before any arithmetic (the kernel is
  // bound by memory latency; on a narrow grid the four are rows, on a wide
  // one parts of a row).  The item counter moves as (ch, j, k) with carries:
  // no division inside the loop.
  constexpr int U = 4;
  const int lane = threadIdx.x & 31;
  const int nch = (L.n[0] + 31) >> 5;
  const long long items = (long long)L.n[1] * L.n[2] * nch;  // < 2^31, checked when the grid is created
  const int W = (gridDim.x * blockDim.x) >> 5;
  const int first = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * U;
  const int stride = W * U;
  int ch = first % nch, j = (first / nch) % L.n[1], k = first / nch / L.n[1];
  const int dch = stride % nch, dj = (stride / nch) % L.n[1], dk = stride / nch / L.n[1];
  for (long long it0 = first; it0 < items; it0 += stride) {
    ST q[U][5], m[U][10];
    bool live[U];
    int cu = ch, ju = j, ku = k;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = cu * 32 + lane;
      live[u] = it0 + u < items && i < L.n[0];
      const long long n = live[u] ? L.at(i, ju, ku) : L.at(0, 0, 0);
#pragma unroll
      for (int v = 0; v < 5; ++v) q[u][v] = Q[v * L.npad + n];
#pragma unroll
      for (int f = 0; f < 10; ++f) m[u][f] = (ST)M[f * L.npad + n];
      if (++cu == nch) {
        cu = 0;
        if (++ju == L.n[1]) { ju = 0; ++ku; }
      }
    }
    ch += dch;
    j += dj;
    k += dk;
    if (ch >= nch) { ch -= nch; ++j; }
    if (j >= L.n[1]) { j -= L.n[1]; ++k; }
    {
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (!live[u]) continue;
        const ST rho = q[u][0], ri = ST(1) / rho;
        const ST uu = q[u][1] * ri, vv = q[u][2] * ri, ww = q[u][3] * ri;
        const ST p = gm1 * (q[u][4] - ST(0.5) * rho * (uu * uu + vv * vv + ww * ww));
        const ST T = g * p * ri;
        const ST c = sqrt(T);
        const ST nu = vfac * sutherland<ST>(mu_inf, s1, T) * ri;
        const ST Jn = m[u][9];
        ST conv = 0, s2 = 0;
#pragma unroll
        for (int kd = 0; kd < 3; ++kd) {
          const ST a = m[u][3 * kd], b = m[u][3 * kd + 1], cc = m[u][3 * kd + 2];
          const ST sq = a * a + b * b + cc * cc;
          conv += Jn * (fabs(a * uu + b * vv + cc * ww) + c * sqrt(sq));
          s2 += sq;
        }
        const ST rate = conv + ST(2) * nu * Jn * Jn * s2;
        best_s = rate > best_s ? rate : best_s;
        if (DIAG) dg.node(q[u], Jn, gm1, g);
      }
    }
  }
  double best = (double)best_s;
  __shared__ double red[RED_THREADS / 32];
  best = warp_max(best);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = best;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = red[0];
    for (int w = 1; w < RED_THREADS / 32; ++w) m = fmax(m, red[w]);
    partial[blockIdx.x] = m;
  }
  __shared__ double sh[DIAG_WORDS][RED_THREADS];
  if (DIAG) {
    double acc[DIAG_WORDS];
    dg.record(acc);
    diag_block_tree(acc, sh);
    if (threadIdx.x == 0)
      for (int c = 0; c < DIAG_WORDS; ++c) partial[RED_BLOCKS + (long long)blockIdx.x * DIAG_WORDS + c] = sh[c][0];
  }
  if (last_block(&sc->count)) {  // max is exact in any order
    if (DIAG) diag_finish(partial + RED_BLOCKS, (int)gridDim.x, sc, sh);
    double m = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) m = fmax(m, ((volatile double*)partial)[b]);
    m = warp_max(m);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 1; w < RED_THREADS / 32; ++w) m = fmax(m, red[w]);
      m = fmax(m, red[0]);
      if (finalize) {
        double dt = cfl / m;
        sc->dt = dt;
        sc->time += dt;
        sc->step += 1;
      } else {
        sc->rate = m;  // the blocks' rates are combined by k_rate_combine
      }
      sc->count = 0;
    }
  }
}

template <typename ST, typename MT, bool DIAG = false>
__global__ void __launch_bounds__(RED_THREADS) k_timestep(Layout L, FlowC F, const ST* __restrict__ Q,
                                                          const MT* __restrict__ M, Scalars* sc, double* partial,
                                                          double cfl, bool finalize) {
  timestep_body<ST, MT, DIAG>(L, F, Q, M, sc, partial, cfl, finalize);
}

// batched: grid blockIdx.y of the table; gridDim.x blocks per grid
struct RateCtx {
  Layout L;
  FlowC F;
  const void* Q0;
  const void* M;
  Scalars* sc;
  double* partial;
};

template <typename ST, typename MT>
__global__ void __launch_bounds__(RED_THREADS) k_timestep_batch(const RateCtx* __restrict__ ctx, double cfl,
                                                                bool finalize) {
  const RateCtx& X = ctx[blockIdx.y];
  timestep_body<ST, MT>(X.L, X.F, (const ST*)X.Q0, (const MT*)X.M, X.sc, X.partial, cfl, finalize);
}

// Blocks of one grid: the grid's rate is the largest of its blocks' (exact
// in any order), and every block takes the one time step it gives.
__global__ void k_rate_combine(const RateCtx* __restrict__ ctx, int n, double cfl) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double m = 0.0;
  for (int b = 0; b < n; ++b) m = fmax(m, ctx[b].sc->rate);
  const double dt = cfl / m;
  for (int b = 0; b < n; ++b) {
    Scalars* sc = ctx[b].sc;
    sc->dt = dt;
    sc->time += dt;
    sc->step += 1;
  }
}

// one block of a grid partitioned over ranks: its rate has been combined with
// the other blocks' (the largest) by the caller
__global__ void k_advance_from_rate(Scalars* sc, double cfl) {
  const double dt = cfl / sc->rate;
  sc->dt = dt;
  sc->time += dt;
  sc->step += 1;
}

__global__ void k_fixed_dt(Scalars* sc, double dt) {
  sc->dt = dt;
  sc->time += dt;
  sc->step += 1;
}

// Diagnostics of the state (records as described above).  Per-node
// arithmetic in the state's type; each lane takes four nodes of its row at a
// time with all their loads issued first.
template <typename ST, typename MT>
__global__ void __launch_bounds__(RED_THREADS) k_diag(Layout L, FlowC F, const ST* __restrict__ Q,
                                                      const MT* __restrict__ M, Scalars* sc, double* partial) {
  const ST gm1 = flow_const<ST>(F.gm1, F.gm1_f), g = flow_const<ST>(F.gamma, F.gamma_f);
  DiagAcc<ST> dg;
  constexpr int U = 4;
  const int lane = threadIdx.x & 31;
  const int W = (gridDim.x * blockDim.x) >> 5;
  const int rows = L.n[1] * L.n[2];
  for (int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < rows; r += W) {
    const long long row = L.at(0, r % L.n[1], r / L.n[1]);
    for (int ib = 0; ib < L.n[0]; ib += 32 * U) {
      ST q[U][5], Jn[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int i = ib + lane + 32 * u;
        const long long n = row + (i < L.n[0] ? i : 0);
#pragma unroll
        for (int v = 0; v < 5; ++v) q[u][v] = Q[(long long)v * L.npad + n];
        Jn[u] = (ST)M[9 * L.npad + n];
      }
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (ib + lane + 32 * u < L.n[0]) dg.node(q[u], Jn[u], gm1, g);
    }
  }
  double acc[DIAG_WORDS];
  dg.record(acc);
  __shared__ double sh[DIAG_WORDS][RED_THREADS];
  diag_block_tree(acc, sh);
  if (threadIdx.x == 0)
    for (int c = 0; c < DIAG_WORDS; ++c) partial[(long long)blockIdx.x * DIAG_WORDS + c] = sh[c][0];
  if (last_block(&sc->dcount)) {
    diag_finish(partial, (int)gridDim.x, sc, sh);
    if (threadIdx.x == 0) sc->dcount = 0;
  }
}

}  // namespace

cudaError_t launch_timestep(const GridDev& g, double cfl, double dt_fixed, cudaStream_t s) {
  if (cfl <= 0.0) {
    if (g.step_diag) {  // the diagnostics of the step's state by their own pass
      cudaError_t e = launch_diagnostics(g, s);
      if (e != cudaSuccess) return e;
    }
    k_fixed_dt<<<1, 1, 0, s>>>(g.sc, dt_fixed);
    count_launches(1);
    return cudaGetLastError();
  }
  const int nb = red_grid(2);
  if (g.step_diag) {
    switch (g.prec) {
      case JZ_P64:
        k_timestep<double, double, true><<<nb, RED_THREADS, 0, s>>>(g.L, g.F, (const double*)g.Q0,
                                                                   (const double*)g.M, g.sc, g.partial, cfl, true);
        break;
      case JZ_P32_M64:
        k_timestep<float, double, true><<<nb, RED_THREADS, 0, s>>>(g.L, g.F, (const float*)g.Q0,
                                                                  (const double*)g.M, g.sc, g.partial, cfl, true);
        break;
      default:
        k_timestep<float, float, true><<<nb, RED_THREADS, 0, s>>>(g.L, g.F, (const float*)g.Q0, (const float*)g.M,
                                                                 g.sc, g.partial, cfl, true);
        break;
    }
    count_launches(1);
    return cudaGetLastError();
  }
  switch (g.prec) {
    case JZ_P64:
      k_timestep<double, double><<<nb, RED_THREADS, 0, s>>>(g.L, g.F, (const double*)g.Q0, (const double*)g.M, g.sc,
                                                            g.partial, cfl, true);
      break;
    case JZ_P32_M64:
      k_timestep<float, double><<<nb, RED_THREADS, 0, s>>>(g.L, g.F, (const float*)g.Q0, (const double*)g.M, g.sc,
                                                           g.partial, cfl, true);
      break;
    default:
      k_timestep<float, float><<<nb, RED_THREADS, 0, s>>>(g.L, g.F, (const float*)g.Q0, (const float*)g.M, g.sc,
                                                          g.partial, cfl, true);
      break;
  }
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_rate(const GridDev& g, cudaStream_t s) {
  switch (g.prec) {
    case JZ_P64:
      k_timestep<double, double><<<red_grid(2), RED_THREADS, 0, s>>>(g.L, g.F, (const double*)g.Q0,
                                                                    (const double*)g.M, g.sc, g.partial, 1.0, false);
      break;
    case JZ_P32_M64:
      k_timestep<float, double><<<red_grid(2), RED_THREADS, 0, s>>>(g.L, g.F, (const float*)g.Q0,
                                                                   (const double*)g.M, g.sc, g.partial, 1.0, false);
      break;
    default:
      k_timestep<float, float><<<red_grid(2), RED_THREADS, 0, s>>>(g.L, g.F, (const float*)g.Q0, (const float*)g.M,
                                                                  g.sc, g.partial, 1.0, false);
      break;
  }
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_advance_from_rate(const GridDev& g, double cfl, cudaStream_t s) {
  k_advance_from_rate<<<1, 1, 0, s>>>(g.sc, cfl);
  count_launches(1);
  return cudaGetLastError();
}

size_t rate_ctx_bytes() { return sizeof(RateCtx); }

void rate_ctx_fill(void* dst, const GridDev& g) {
  RateCtx& X = *(RateCtx*)dst;
  X.L = g.L;
  X.F = g.F;
  X.Q0 = g.Q0;
  X.M = g.M;
  X.sc = g.sc;
  X.partial = g.partial;
}

cudaError_t launch_timestep_batch(int prec, const void* ctx, int n, double cfl, bool coupled, cudaStream_t s) {
  const dim3 grid(64, n);  // 64 blocks per grid (partials hold RED_BLOCKS)
  const RateCtx* X = (const RateCtx*)ctx;
  const bool fin = !coupled;
  switch (prec) {
    case JZ_P64: k_timestep_batch<double, double><<<grid, RED_THREADS, 0, s>>>(X, cfl, fin); break;
    case JZ_P32_M64: k_timestep_batch<float, double><<<grid, RED_THREADS, 0, s>>>(X, cfl, fin); break;
    default: k_timestep_batch<float, float><<<grid, RED_THREADS, 0, s>>>(X, cfl, fin); break;
  }
  count_launches(1);
  if (coupled) {
    k_rate_combine<<<1, 32, 0, s>>>(X, n, cfl);
    count_launches(1);
  }
  return cudaGetLastError();
}

cudaError_t launch_diagnostics(const GridDev& g, cudaStream_t s) {
  switch (g.prec) {
    case JZ_P64:
      k_diag<double, double><<<red_grid(3), RED_THREADS, 0, s>>>(g.L, g.F, (const double*)g.Q0, (const double*)g.M,
                                                                g.sc, g.partial);
      break;
    case JZ_P32_M64:
      k_diag<float, double><<<red_grid(3), RED_THREADS, 0, s>>>(g.L, g.F, (const float*)g.Q0, (const double*)g.M,
                                                               g.sc, g.partial);
      break;
    default:
      k_diag<float, float><<<red_grid(3), RED_THREADS, 0, s>>>(g.L, g.F, (const float*)g.Q0, (const float*)g.M, g.sc,
                                                              g.partial);
      break;
  }
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace jz
