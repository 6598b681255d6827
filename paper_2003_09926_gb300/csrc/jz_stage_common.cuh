// jz_stage_common.cuh -- pieces shared by the scalar and the vector-record
// fused stage kernels: ring record layout, flow constants in the arithmetic
// type, elementary-function choices, TMA / mbarrier helpers (inline PTX), the
// per-grid kernel context and the per-launch stage selection.
#pragma once

#include <cmath>
#include <cstdint>

#include "jz_fastmath.cuh"
#include "jz_internal.h"

namespace jz {
namespace stg {

// ring record
enum { V_RHO = 0, V_U = 1, V_V = 2, V_W = 3, V_E = 4, V_P = 5, V_T = 6, NV = 7 };

template <typename R>
struct KConst {
  R gamma, gm1, cp, mu_inf, s1, s1p1, inv_pr, inv_prt, cs2, k2, k4, sigma;
  int viscous, sgs, sig_half;
  int vreman;  // eddy viscosity of Vreman's model instead of Smagorinsky's
};

template <typename R>
__host__ __device__ inline KConst<R> make_kconst(const FlowC& F) {
  KConst<R> c;
  c.gamma = (R)F.gamma;
  c.gm1 = (R)F.gm1;
  c.cp = (R)F.cp;
  c.mu_inf = (R)F.mu_inf;
  c.s1 = (R)F.s1;
  c.s1p1 = (R)(1.0 + F.s1);
  c.inv_pr = (R)(1.0 / F.pr);
  c.inv_prt = (R)(1.0 / F.prt);
  c.cs2 = (R)(F.cs * F.cs);
  c.k2 = (R)F.k2;
  c.k4 = (R)F.k4;
  c.sigma = (R)F.sigma;
  c.viscous = F.viscous;
  c.sgs = F.cs > 0.0;
  c.sig_half = F.sigma == 0.5;
  c.vreman = F.sgs == JZ_SGS_VREMAN;
  return c;
}

template <typename R>
__device__ __forceinline__ R rmax(R a, R b) { return a > b ? a : b; }

// Flow models that the FP32 vector-record stage kernel is compiled for with
// constant flags: the stage body of each model carries no branch on the
// flags of the others, so that the compiler schedules the viscous, eddy
// viscosity and dissipation arithmetic of a node as one block.  The runtime
// model reads the flags of KConst and serves every other combination; the
// arithmetic of a node is the same expression in every build.
constexpr int kModelRuntime = 0;      // flags read at run time
constexpr int kModelSmagorinsky = 1;  // viscous, Smagorinsky eddy viscosity, sigma = 1/2
constexpr int kModelVreman = 2;       // viscous, Vreman eddy viscosity, sigma = 1/2
constexpr int kModelEuler = 3;        // inviscid, sigma = 1/2
constexpr int kModels = 4;

template <typename R>
__host__ __device__ inline int flow_model(const KConst<R>& c) {
  if (!c.sig_half) return kModelRuntime;
  if (!c.viscous) return kModelEuler;
  if (!c.sgs) return kModelRuntime;
  return c.vreman ? kModelVreman : kModelSmagorinsky;
}

// The flags of model MD: compile-time constants, except for the runtime model.
template <int MD>
struct ModelFlags {
  template <typename R>
  static __device__ __forceinline__ bool viscous(const KConst<R>& c) {
    return MD == kModelRuntime ? c.viscous != 0 : MD != kModelEuler;
  }
  template <typename R>
  static __device__ __forceinline__ bool sgs(const KConst<R>& c) {
    return MD == kModelRuntime ? c.sgs != 0 : MD != kModelEuler;
  }
  template <typename R>
  static __device__ __forceinline__ bool sig_half(const KConst<R>& c) {
    return MD == kModelRuntime ? c.sig_half != 0 : true;
  }
  // eddy viscosity model: -1 read at run time, 0 Smagorinsky, 1 Vreman
  static constexpr int eddy = MD == kModelRuntime ? -1 : (MD == kModelVreman ? 1 : 0);
};

// Eddy viscosity mu_t / rho from the velocity gradients g[a][m] = du_a/dx_m
// and J (Delta^2 = J^(-2/3)).
//   Smagorinsky: (C_s Delta)^2 |S|, |S| = sqrt(2 S_ij S_ij).
//   Vreman (2004): c Delta^2 sqrt(B / (g_am g_am)), c = 2.5 C_s^2, with
//     b_ab = sum_m g[a][m] g[b][m] and B = b00 b11 - b01^2 + b00 b22 - b02^2
//     + b11 b22 - b12^2 (the sum of b's principal 2x2 minors, >= 0; clamped at
//     0 against rounding); 0 where all gradients vanish (g_am g_am = 0).
//     B <= (g_am g_am)^2/3, so the model tends to 0 with the gradients.  In
//     FP32 the reciprocal flushes subnormal operands to zero, so there the
//     model is also taken as 0 where g_am g_am is below the smallest normal
//     FP32 number; FP64 uses the plain > 0 test.
// EDDY: -1 the model of c (read at run time), 0 Smagorinsky, 1 Vreman.
template <typename R, int EDDY = -1>
__device__ __forceinline__ R eddy_nu(const KConst<R>& c, const R g[4][3], R Jn) {
  if (EDDY < 0 ? c.vreman != 0 : EDDY == 1) {
    const R tiny = sizeof(R) == 4 ? R(1.17549435e-38f) : R(0);
    R b[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int d = a; d < 3; ++d) b[a][d] = g[a][0] * g[d][0] + g[a][1] * g[d][1] + g[a][2] * g[d][2];
    const R aa = b[0][0] + b[1][1] + b[2][2];
    const R B = b[0][0] * b[1][1] - b[0][1] * b[0][1] + b[0][0] * b[2][2] - b[0][2] * b[0][2] +
                b[1][1] * b[2][2] - b[1][2] * b[1][2];
    if (!(aa > tiny)) return R(0);
    return R(2.5) * c.cs2 * Fn<R>::jm23(Jn) * Fn<R>::sqrt_(Fn<R>::div(rmax(B, R(0)), aa));
  }
  const R s12 = R(0.5) * (g[0][1] + g[1][0]), s13 = R(0.5) * (g[0][2] + g[2][0]);
  const R s23 = R(0.5) * (g[1][2] + g[2][1]);
  const R ss = g[0][0] * g[0][0] + g[1][1] * g[1][1] + g[2][2] * g[2][2] + R(2) * (s12 * s12 + s13 * s13 + s23 * s23);
  return c.cs2 * Fn<R>::sqrt_(R(2) * ss) * Fn<R>::jm23(Jn);
}

// ---------------------------------------------------------------------------
// TMA and mbarrier helpers (inline PTX, sm_90+ async proxy)
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_async_shared() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait: gives up after `limit` SM cycles (by default 2^31, about a
// second).
constexpr long long kWaitLimit = 1LL << 31;
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, long long limit = kWaitLimit) {
  const long long start = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - start > limit) return false;
  }
  return true;
}

// Explicit completion of `bytes` transaction bytes on the barrier's current
// phase (used only by the stall test's recovery, see StageSel::stall).
__device__ __forceinline__ void mbar_complete_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.complete_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

// 4-D tiled TMA load: box at (x, y, z, w) of the tensor map into shared memory.
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y, int z,
                                            int w) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
      "[%6];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(w), "r"(smem_addr(bar))
      : "memory");
}

// Everything the stage kernel needs about one grid: TMA maps of the three
// state copies and of the metrics, layout, state pointers, device scalars
// (time step), flow constants and the k-chunk length.  Passed as a kernel
// parameter for one grid, or read from a device table for a batch.
template <typename R, typename MT>
struct alignas(128) StageCtx {
  CUtensorMap tmQ[3];  // Q0, QA, QB
  CUtensorMap tmM;     // metrics
  CUtensorMap tmMv;    // metrics, box of the tile plus a one-node halo (FP32 record kernel)
  CUtensorMap tmQ0u;   // Q0, box of the tile rows (FP32 record kernel's update)
  Layout L;
  R* Q[3];             // Q0, QA, QB
  double* Q0d;         // FP64 state between steps (JZ_P32_S64; else null)
  const Scalars* sc;
  int* err;            // sticky error flag (bounded-wait timeout)
  FlowC F;
  KConst<R> k;         // flow constants in the arithmetic type, prepared on the host
  int kc;
};

// Per-launch stage selection: alpha_l, input copy Q^(l-1), output copy Q^(l).
// stall (test only, 0 otherwise): every TMA copy of the launch expects
// kStallBytes more than it delivers, so its barrier phase cannot complete,
// and waits give up after kStallLimit cycles.  The kernel then takes its
// timeout path: it records the failure, completes the missing bytes itself,
// waits (default limit) for the real copies to land and returns.
struct StageSel {
  double alpha;
  int qin, qout;
  int stall;
};
constexpr uint32_t kStallBytes = 16;
constexpr long long kStallLimit = 1LL << 16;

__device__ __forceinline__ void init_barriers(uint64_t* bar) {
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_init(&bar[2], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
}

// after a timeout: record it and let this CTA's copies still in flight land
// (xtx: the transaction bytes each copy expects beyond what it delivers,
// nonzero only in the stall test, completed here before the wait)
__device__ __forceinline__ void drain_after_timeout(uint64_t* bar, int* err, const int issued[3],
                                                    const int waited[3], uint32_t xtx) {
  if (threadIdx.x == 0) {
    atomicExch(err, 1);
    for (int b = 0; b < 3; ++b)
      for (int u = waited[b]; u < issued[b]; ++u) {
        if (xtx) mbar_complete_tx(&bar[b], xtx);
        if (!mbar_wait_bounded(&bar[b], u & 1)) break;  // phase u of barrier b
      }
  }
  __syncthreads();
}

constexpr double kRkAlpha[5] = {1.0 / 4.0, 1.0 / 6.0, 3.0 / 8.0, 1.0 / 2.0, 1.0};

}  // namespace stg

// CTAs per SM of the FP32 vector-record kernel for a tile shape: tiles of at
// most 256 nodes (16 x 16) run two CTAs per SM (320 threads, <= 113 KB of
// shared memory each), larger tiles one
constexpr int vr_ctas_per_sm(int ti, int tj) { return ti * tj <= 256 ? 2 : 1; }

// FP32 kernel with vector node records (jz_stage_v.cu, one build per tile shape)
#define JZ_STAGE_V_DECL(S)                                                                                    \
  cudaError_t stage_v_configure_##S();                                                                        \
  cudaError_t launch_stage_v_##S(const stg::StageCtx<float, float>& X, const stg::StageSel& st, cudaStream_t s); \
  cudaError_t launch_stage_v_batch_##S(const void* ctx, const int4* items, int nitems, unsigned int* queue,      \
                                       const stg::StageSel& st, int model, cudaStream_t s);
JZ_STAGE_V_DECL(32x16)
JZ_STAGE_V_DECL(16x32)
JZ_STAGE_V_DECL(16x16)
#undef JZ_STAGE_V_DECL
}  // namespace jz
