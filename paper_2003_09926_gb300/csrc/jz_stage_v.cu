// jz_stage_v.cu -- the FP32 fused Runge-Kutta stage kernel with vector node
// records: residual evaluation and stage update in one pass over HBM.
//
// Paper: arXiv 2003.09926, Section 3 and Section 4.2: per Runge-Kutta
// sub-step, the centred inviscid flux in general curvilinear coordinates, the
// Turkel-Vatsa anisotropic scalar artificial dissipation (pressure sensor,
// five-point stencil, Section 4.3), the viscous flux (Stokes stress, Fourier
// heat flux, Sutherland viscosity) plus a Smagorinsky (or Vreman) eddy viscosity, then
// the update Q^(l) = Q^(0) - alpha_l dt J R(Q^(l-1)) of the 5-stage scheme.
// The residual is taken in face form, R_n = sum_k (h^k_{n+1/2} - h^k_{n-1/2})
// with h_{n+1/2} = (G_n + G_{n+1})/2 - d_{n+1/2}, G = E - F the contravariant
// inviscid minus viscous flux: the paper's central difference plus
// dissipation, telescoping exactly.
//
// Organisation (2.5-D streaming over a TI x TJ (i, j) tile and a chunk of
// k-planes; the file is compiled once per tile shape the autotuner chooses
// from: 16 x 16 (the default, two CTAs per SM), 32 x 16 and 16 x 32 (one CTA
// per SM), VR_TI / VR_TJ, and its entry points carry the shape in their
// names; within a shape, once per flow model with the model's flags as
// constants plus once with the flags read at run time, and within a build
// once per node role):
//  - TMA stages the conserved variables of one plane (tile plus a two-node
//    halo) into a planar buffer, and the metric fields of one plane (tile
//    plus a one-node halo) into a second buffer; waits are bounded;
//  - each staged plane is converted once into two rings of node records:
//    conserved (rho, rho u, rho v, rho w | e) over four planes and primitive
//    (u, v, w, T | p) over three, each a float4 plus a float, so that a
//    node's stencil values arrive with two shared-memory loads;
//  - one thread per node of the plus-shaped set (tile nodes plus the
//    one-node i and j halo) forms G^k, the dissipation radius lambda~^k and
//    the sensor nu^k of its node (tile threads in all three directions, halo
//    threads in their own direction);
//  - i and j face fluxes go through shared memory as float4 + float records,
//    the k face flux of a column stays in its thread's registers;
//  - two block barriers per plane: node pass of plane t+1, k face, i/j
//    residual and update of plane t | i/j face fluxes of plane t+1 and the
//    conversion of the plane three ahead.
#include <cmath>
#include <cstdint>

#include "jz_stage_common.cuh"

#ifndef VR_TI
#define VR_TI 32
#define VR_TJ 16
#endif
// face fluxes, node gradients and contravariant viscous fluxes on packed
// FP32x2 component pairs
#ifndef VR_PACKED_FACES
#define VR_PACKED_FACES 1
#endif
#define VR_CAT3(a, b, c) a##_##b##x##c
#define VR_CAT(a, b, c) VR_CAT3(a, b, c)
#define VR_FN(name) VR_CAT(name, VR_TI, VR_TJ)

namespace jz {

using namespace stg;

namespace {

namespace vr {
constexpr int TI = VR_TI, TJ = VR_TJ;
constexpr int MINB = vr_ctas_per_sm(TI, TJ);    // CTAs per SM
constexpr int NTILE = TI * TJ;                  // tile nodes
constexpr int NJH = 2 * TI, NIH = 2 * TJ;       // j-halo (rows -1, TJ) and i-halo (columns -1, TI) nodes
constexpr int NT = NTILE + NJH + NIH;           // threads (608 for 32 x 16 and 16 x 32)
static_assert(NT % 32 == 0, "whole warps");
constexpr int NCH = 3 * (NJH + NIH);            // plane elements converted by the halo threads
constexpr int RW = TI + 4, RH = TJ + 4, PL = RW * RH;  // staged plane: tile + two-node halo (36 x 20)
constexpr int MH = TJ + 2, MPL = RW * MH;        // metric box: rows -1 .. TJ, 36 columns
// Warp layout of the tile threads.  A warp holds 32 nodes: a full row of a
// 32-wide tile, or two rows of a 16-wide tile.  In the 16 x 16 build the two
// rows of a warp are r and r + 4 (warps 0-3: rows 0-3 and 4-7, warps 4-7:
// rows 8-11 and 12-15), and every per-row buffer has a row stride of 20
// words, so the two half-warps of a scalar shared-memory access sit 80 = 16
// (mod 32) banks apart and never conflict.
constexpr bool ROWS4 = TI == 16 && TJ == 16;
// ring records: rows padded to 37 so that the column-wise accesses of the
// i-halo warp fall on distinct banks (unpadded rows of 20 in the 16 x 16
// build, for the warp layout above)
constexpr int RR = ROWS4 ? RW : RW + 1, RPL = RR * RH;
// ring depths (planes): conserved records 4 (the k face t + 1/2 reads
// planes t-1 .. t+2), primitive records 3 (the node pass of plane t reads
// planes t-1 .. t+1)
constexpr int NSQ = 4, NSP = 3;
// node buffers: columns -1..TI / rows -1..TJ; face buffers: i faces 0..TI /
// j faces 0..TJ.  The i-direction rows are padded (distinct banks for the
// i-halo warp's column accesses; a stride of 20 in the 16 x 16 build).
constexpr int GIW = ROWS4 ? TI + 4 : TI + 3, GJH = TJ + 2;
constexpr int HIW = ROWS4 ? TI + 4 : TI + 3, HJH = TJ + 1;
constexpr size_t al(size_t x) { return (x + 127) / 128 * 128; }
constexpr size_t RAW_B = al(4 * 5 * PL);
constexpr size_t QV_B = al(16 * NSQ * RPL), QE_B = al(4 * NSQ * RPL);
constexpr size_t PV_B = al(16 * NSP * RPL), PP_B = al(4 * NSP * RPL);
constexpr size_t MET_B = al(4 * 10 * MPL);
constexpr int UPL = RW * TJ;                     // Q^(0) box: tile rows, 36 columns
constexpr size_t Q0_B = al(4 * 5 * UPL);
constexpr size_t GI4_B = al(16 * TJ * GIW), GI1_B = al(4 * TJ * GIW);
// the scalar part of the j-direction records: rows of 20 in the 16 x 16 build
// (the float4 / float2 parts are conflict-free at any row stride)
constexpr int JS1 = ROWS4 ? TI + 4 : TI;
constexpr size_t GJ4_B = al(16 * GJH * TI), GJ1_B = al(4 * GJH * JS1);
constexpr size_t LI_B = al(8 * TJ * GIW), LJ_B = al(8 * GJH * TI);
constexpr size_t HI4_B = al(16 * TJ * HIW), HI1_B = al(4 * TJ * HIW);
constexpr size_t HJ4_B = al(16 * HJH * TI), HJ1_B = al(4 * HJH * JS1);
constexpr size_t O_RAW = 0;
constexpr size_t O_QV = O_RAW + RAW_B;
constexpr size_t O_QE = O_QV + QV_B;
constexpr size_t O_PV = O_QE + QE_B;
constexpr size_t O_PP = O_PV + PV_B;
constexpr size_t O_MET = O_PP + PP_B;
constexpr size_t O_Q0 = O_MET + MET_B;
constexpr size_t O_GI4 = O_Q0 + Q0_B;
constexpr size_t O_GI1 = O_GI4 + GI4_B;
constexpr size_t O_GJ4 = O_GI1 + GI1_B;
constexpr size_t O_GJ1 = O_GJ4 + GJ4_B;
constexpr size_t O_LI = O_GJ1 + GJ1_B;
constexpr size_t O_LJ = O_LI + LI_B;
constexpr size_t O_HI4 = O_LJ + LJ_B;
constexpr size_t O_HI1 = O_HI4 + HI4_B;
constexpr size_t O_HJ4 = O_HI1 + HI1_B;
constexpr size_t O_HJ1 = O_HJ4 + HJ4_B;
constexpr size_t O_BAR = O_HJ1 + HJ1_B;
constexpr size_t BYTES = O_BAR + 128;
// during a chunk's prologue three more raw planes are staged over the node
// and face buffers, which are not in use yet
constexpr size_t O_SCR = O_GI4;
static_assert(O_BAR - O_SCR >= 3 * RAW_B, "prologue staging does not fit");
static_assert(BYTES <= 232448, "shared memory");
// two CTAs per SM: 228 KB per SM, 1 KB reserved per CTA, a few bytes of
// static shared memory in the batched kernel
static_assert(MINB == 1 || 2 * (BYTES + 128 + 1024) <= 228 * 1024, "two CTAs per SM do not fit");
constexpr uint32_t RAW_TX = 4 * 5 * PL;
constexpr uint32_t MET_TX = 4 * 10 * MPL;
constexpr uint32_t Q0_TX = 4 * 5 * UPL;
// mbarriers: 0 raw buffer, 1..3 prologue staging, 4 metrics, 5 Q^(0)
constexpr int B_RAW = 0, B_MET = 4, B_Q0 = 5, NBAR = 6;
}  // namespace vr

__device__ __forceinline__ void ld5(const float4* v4, const float* v1, int i, float q[5]) {
  const float4 a = v4[i];
  q[0] = a.x; q[1] = a.y; q[2] = a.z; q[3] = a.w;
  q[4] = v1[i];
}
__device__ __forceinline__ void st5(float4* v4, float* v1, int i, const float q[5]) {
  v4[i] = make_float4(q[0], q[1], q[2], q[3]);
  v1[i] = q[4];
}
// a record whose two parts have different row strides: row y, column x
__device__ __forceinline__ void ld5j(const float4* v4, const float* v1, int y, int x, float q[5]) {
  const float4 a = v4[y * vr::TI + x];
  q[0] = a.x; q[1] = a.y; q[2] = a.z; q[3] = a.w;
  q[4] = v1[y * vr::JS1 + x];
}
__device__ __forceinline__ void st5j(float4* v4, float* v1, int y, int x, const float q[5]) {
  v4[y * vr::TI + x] = make_float4(q[0], q[1], q[2], q[3]);
  v1[y * vr::JS1 + x] = q[4];
}
__device__ __forceinline__ void mbar_inval(uint64_t* bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}
// bounded wait with a fast path (the copy has normally landed long before)
__device__ __forceinline__ bool wait_v(uint64_t* bar, uint32_t parity, long long limit) {
  return mbar_try_wait(bar, parity) || mbar_wait_bounded(bar, parity, limit);
}

// Node quantities of node (x, y) of plane kk: G^k = E^k - F^k, lambda~^k,
// nu^k.  Primitive records of the planes below / at / above in slots sM, sC,
// sP; the conserved record of the plane in slot qC.  DIR = 0: all three
// directions; DIR = 1 / 2 / 3: direction i / j / k only.
template <int DIR, int MD>
__device__ __forceinline__ void node_v(const float4* __restrict__ PV, const float* __restrict__ PP,
                                       const float4* __restrict__ QV, const float* __restrict__ QE,
                                       const float* __restrict__ met, int sM, int sC, int sP, int qC, int x, int y,
                                       const KConst<float>& c, float G[3][5], float lt[3], float nu[3], float& Jn) {
  using namespace vr;
  const int o = (y + 2) * RR + x + 2;
  const int mo = (y + 1) * RW + x + 2;
  float S[9];
#pragma unroll
  for (int f = 0; f < 9; ++f) S[f] = met[f * MPL + mo];
  Jn = met[9 * MPL + mo];
  const float4* pc = PV + sC;
  const float4 r0 = pc[o];
  const float u = r0.x, v = r0.y, w = r0.z, T = r0.w;
  const float p = PP[sC + o];
  const float rho = QV[qC + o].x;
  const float e = QE[qC + o];
  constexpr int K0 = DIR == 0 ? 0 : DIR - 1;  // DIR 3: direction k only
  constexpr int K1 = DIR == 0 ? 3 : DIR;

  float Fv[3][4];  // viscous flux vectors F_m (m = x, y, z), components 1..4
#pragma unroll
  for (int m = 0; m < 3; ++m)
#pragma unroll
    for (int q = 0; q < 4; ++q) Fv[m][q] = 0.f;
  if (ModelFlags<MD>::viscous(c)) {
    // Cartesian gradients of u, v, w, T: J/2 sum_k S^k_m (phi_+ - phi_-)
    const float4 a0 = pc[o + 1], b0 = pc[o - 1], a1 = pc[o + RR], b1 = pc[o - RR];
    const float4 a2 = PV[sP + o], b2 = PV[sM + o];
    const float hJ = 0.5f * Jn;
    float g[4][3];
#if VR_PACKED_FACES
    {  // the same sums on the variable pairs (u, v) and (w, T), packed FP32x2
      const float2 m1 = make_float2(-1.f, -1.f), h2 = make_float2(hJ, hJ);
      const float2 d0[2] = {__ffma2_rn(make_float2(b0.x, b0.y), m1, make_float2(a0.x, a0.y)),
                            __ffma2_rn(make_float2(b0.z, b0.w), m1, make_float2(a0.z, a0.w))};
      const float2 d1[2] = {__ffma2_rn(make_float2(b1.x, b1.y), m1, make_float2(a1.x, a1.y)),
                            __ffma2_rn(make_float2(b1.z, b1.w), m1, make_float2(a1.z, a1.w))};
      const float2 d2[2] = {__ffma2_rn(make_float2(b2.x, b2.y), m1, make_float2(a2.x, a2.y)),
                            __ffma2_rn(make_float2(b2.z, b2.w), m1, make_float2(a2.z, a2.w))};
#pragma unroll
      for (int pq = 0; pq < 2; ++pq)
#pragma unroll
        for (int m = 0; m < 3; ++m) {
          float2 t = __fmul2_rn(make_float2(S[m], S[m]), d0[pq]);
          t = __ffma2_rn(make_float2(S[3 + m], S[3 + m]), d1[pq], t);
          t = __ffma2_rn(make_float2(S[6 + m], S[6 + m]), d2[pq], t);
          t = __fmul2_rn(h2, t);
          g[2 * pq][m] = t.x;
          g[2 * pq + 1][m] = t.y;
        }
    }
#else
    const float d0[4] = {a0.x - b0.x, a0.y - b0.y, a0.z - b0.z, a0.w - b0.w};
    const float d1[4] = {a1.x - b1.x, a1.y - b1.y, a1.z - b1.z, a1.w - b1.w};
    const float d2[4] = {a2.x - b2.x, a2.y - b2.y, a2.z - b2.z, a2.w - b2.w};
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int m = 0; m < 3; ++m) g[q][m] = hJ * (S[m] * d0[q] + S[3 + m] * d1[q] + S[6 + m] * d2[q]);
#endif
    const float mu = Fn<float>::div(c.mu_inf * T * Fn<float>::sqrt_(T) * c.s1p1, T + c.s1);  // Sutherland
    float mu_t = 0.f;
    // Smagorinsky or Vreman, Delta = J^(-1/3); an unfused product, so that
    // mu + mu_t rounds alike in the constant-flag and runtime-flag builds
    if (ModelFlags<MD>::sgs(c)) mu_t = Fn<float>::mul_rn(rho, eddy_nu<float, ModelFlags<MD>::eddy>(c, g, Jn));
    const float mue = mu + mu_t;
    const float kap = c.cp * (mu * c.inv_pr + mu_t * c.inv_prt);
    const float div3 = (g[0][0] + g[1][1] + g[2][2]) * (2.f / 3.f);
    const float t01 = mue * (g[0][1] + g[1][0]), t02 = mue * (g[0][2] + g[2][0]), t12 = mue * (g[1][2] + g[2][1]);
    Fv[0][0] = mue * (2.f * g[0][0] - div3); Fv[0][1] = t01; Fv[0][2] = t02;
    Fv[1][0] = t01; Fv[1][1] = mue * (2.f * g[1][1] - div3); Fv[1][2] = t12;
    Fv[2][0] = t02; Fv[2][1] = t12; Fv[2][2] = mue * (2.f * g[2][2] - div3);
#pragma unroll
    for (int m = 0; m < 3; ++m) Fv[m][3] = u * Fv[m][0] + v * Fv[m][1] + w * Fv[m][2] + kap * g[3][m];
  }

  float lam[3], U[3];
  const float cson = Fn<float>::sqrt_(T);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    U[k] = S[3 * k] * u + S[3 * k + 1] * v + S[3 * k + 2] * w;
    const float sn = Fn<float>::sqrt_(S[3 * k] * S[3 * k] + S[3 * k + 1] * S[3 * k + 1] + S[3 * k + 2] * S[3 * k + 2]);
    lam[k] = fabsf(U[k]) + cson * sn;
  }
  float sq[3] = {0.f, 0.f, 0.f};
  if (ModelFlags<MD>::sig_half(c)) {
#pragma unroll
    for (int k = 0; k < 3; ++k) sq[k] = Fn<float>::sqrt_(lam[k]);
  }
  const float m1 = rho * u, m2 = rho * v, m3 = rho * w;
#pragma unroll
  for (int k = K0; k < K1; ++k) {
    const float Sx = S[3 * k], Sy = S[3 * k + 1], Sz = S[3 * k + 2];
    float Fk[4];
#if VR_PACKED_FACES
#pragma unroll
    for (int q = 0; q < 4; q += 2) {
      float2 t = __fmul2_rn(make_float2(Sx, Sx), make_float2(Fv[0][q], Fv[0][q + 1]));
      t = __ffma2_rn(make_float2(Sy, Sy), make_float2(Fv[1][q], Fv[1][q + 1]), t);
      t = __ffma2_rn(make_float2(Sz, Sz), make_float2(Fv[2][q], Fv[2][q + 1]), t);
      Fk[q] = t.x;
      Fk[q + 1] = t.y;
    }
#else
#pragma unroll
    for (int q = 0; q < 4; ++q) Fk[q] = Sx * Fv[0][q] + Sy * Fv[1][q] + Sz * Fv[2][q];
#endif
    // E^k = [rho U, rho u U + S_x p, rho v U + S_y p, rho w U + S_z p, (e + p) U]
    G[k][0] = rho * U[k];
    G[k][1] = m1 * U[k] + Sx * p - Fk[0];
    G[k][2] = m2 * U[k] + Sy * p - Fk[1];
    G[k][3] = m3 * U[k] + Sz * p - Fk[2];
    G[k][4] = (e + p) * U[k] - Fk[3];
    const int a = (k + 1) % 3, b = (k + 2) % 3;
    if (ModelFlags<MD>::sig_half(c))  // lambda (1 + (la/l)^1/2 + (lb/l)^1/2) = lambda + sqrt(lambda) (sqrt(la) + sqrt(lb))
      lt[k] = lam[k] + sq[k] * (sq[a] + sq[b]);
    else
      lt[k] = lam[k] > 0.f ? lam[k] * (1.f + Fn<float>::powp(Fn<float>::div(lam[a], lam[k]), c.sigma) +
                                       Fn<float>::powp(Fn<float>::div(lam[b], lam[k]), c.sigma))
                           : 0.f;  // zero face metric (a centreline): the limit for sigma < 1
    float pm, pp;
    if (k == 0) { pm = PP[sC + o - 1]; pp = PP[sC + o + 1]; }
    else if (k == 1) { pm = PP[sC + o - RR]; pp = PP[sC + o + RR]; }
    else { pm = PP[sM + o]; pp = PP[sP + o]; }
    nu[k] = Fn<float>::div(fabsf(pp - 2.f * p + pm), pp + 2.f * p + pm);
  }
}

// dissipative face flux between nodes a and b of a line m, a, b, p:
// h = (Ga + Gb)/2 - lam [e2 (qb - qa) - e4 (qp - 3 qb + 3 qa - qm)],
// lam = (lt_a + lt_b)/2, e2 = k2 max(nu_a, nu_b), e4 = max(0, k4 - e2)
__device__ __forceinline__ void face_v(const KConst<float>& c, float2 La, float2 Lb, const float Ga[5],
                                       const float Gb[5], const float qm[5], const float qa[5], const float qb[5],
                                       const float qp[5], float h[5]) {
  const float lam = 0.5f * (La.x + Lb.x);
  const float e2 = c.k2 * fmaxf(La.y, Lb.y);
  const float e4 = fmaxf(0.f, c.k4 - e2);
  const float l2 = lam * e2, l4 = lam * e4;
#if VR_PACKED_FACES
  // h = (Ga + Gb)/2 - l2 d1 + l4 d3 on component pairs (0, 1) and (2, 3)
  // with packed FP32x2 operations (each lane rounds as its scalar
  // counterpart), component 4 in scalar form
  const float2 m1 = make_float2(-1.f, -1.f), m3 = make_float2(-3.f, -3.f), hf = make_float2(0.5f, 0.5f);
  const float2 ml2 = make_float2(-l2, -l2), pl4 = make_float2(l4, l4);
#pragma unroll
  for (int v = 0; v < 4; v += 2) {
    const float2 a = make_float2(qa[v], qa[v + 1]), b = make_float2(qb[v], qb[v + 1]);
    const float2 m = make_float2(qm[v], qm[v + 1]), p = make_float2(qp[v], qp[v + 1]);
    const float2 d1 = __ffma2_rn(a, m1, b);                       // qb - qa
    const float2 d3 = __ffma2_rn(d1, m3, __ffma2_rn(m, m1, p));  // (qp - qm) - 3 d1
    const float2 g = __fmul2_rn(hf, __fadd2_rn(make_float2(Ga[v], Ga[v + 1]), make_float2(Gb[v], Gb[v + 1])));
    const float2 r = __ffma2_rn(pl4, d3, __ffma2_rn(ml2, d1, g));
    h[v] = r.x;
    h[v + 1] = r.y;
  }
  {
    const float d1 = qb[4] - qa[4];
    const float d3 = (qp[4] - qm[4]) - 3.f * d1;
    h[4] = fmaf(l4, d3, fmaf(-l2, d1, 0.5f * (Ga[4] + Gb[4])));
  }
#else
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    const float d1 = qb[v] - qa[v];
    const float d3 = (qp[v] - qm[v]) - 3.f * d1;
    h[v] = 0.5f * (Ga[v] + Gb[v]) - (l2 * d1 - l4 * d3);
  }
#endif
}

struct Smem {
  float* raw;
  float4* QV;
  float* QE;
  float4* PV;
  float* PP;
  float* met;
  float4 *Gi4, *Gj4, *Hi4, *Hj4;
  float *Gi1, *Gj1, *Hi1, *Hj1;
  float2 *Li, *Lj;
  uint64_t* bar;
  __device__ explicit Smem(unsigned char* s) {
    using namespace vr;
    raw = reinterpret_cast<float*>(s + O_RAW);
    QV = reinterpret_cast<float4*>(s + O_QV);
    QE = reinterpret_cast<float*>(s + O_QE);
    PV = reinterpret_cast<float4*>(s + O_PV);
    PP = reinterpret_cast<float*>(s + O_PP);
    met = reinterpret_cast<float*>(s + O_MET);
    Gi4 = reinterpret_cast<float4*>(s + O_GI4);
    Gi1 = reinterpret_cast<float*>(s + O_GI1);
    Gj4 = reinterpret_cast<float4*>(s + O_GJ4);
    Gj1 = reinterpret_cast<float*>(s + O_GJ1);
    Li = reinterpret_cast<float2*>(s + O_LI);
    Lj = reinterpret_cast<float2*>(s + O_LJ);
    Hi4 = reinterpret_cast<float4*>(s + O_HI4);
    Hi1 = reinterpret_cast<float*>(s + O_HI1);
    Hj4 = reinterpret_cast<float4*>(s + O_HJ4);
    Hj1 = reinterpret_cast<float*>(s + O_HJ1);
    bar = reinterpret_cast<uint64_t*>(s + O_BAR);
  }
};

// A thread's own node data of one plane, kept in registers from the node
// pass to the face pass.
struct Own {
  float Gi[5], Gj[5];  // node fluxes G^i, G^j
  float2 Li, Lj;       // (lambda~, nu) in i and j
};

// Node role of thread tid (warps hold one role each): 0 tile node, 2 j-halo
// node, 1 i-halo node.
__device__ __forceinline__ int role_of(int tid) {
  return tid < vr::NTILE ? 0 : (tid < vr::NTILE + vr::NJH ? 2 : 1);
}

// One work item: tile (bx, by), k-chunk bz of grid X, stage st, for the
// threads of node role ROLE (each role runs its own instantiation of the
// plane march, without branches on the role; all roles pass the same
// sequence of block barriers).  The CTA's
// mbarriers are (re)initialised at the start of every item, so the parity of
// every wait follows from the plane index.  On a bounded-wait timeout the
// item records where it gave up, lets its copies in flight land and returns
// false.
template <int MD, int ROLE>
__device__ __forceinline__ bool item_v(const StageCtx<float, float>& X, const StageSel& st, int bx, int by, int bz,
                                       unsigned char* smem, bool first) {
  using namespace vr;
  Smem sm(smem);
  const Layout& L = X.L;
  const KConst<float> c = X.k;
  const int tid = threadIdx.x;
  const int i0 = bx * TI, j0 = by * TJ;
  const int t0 = L.lo[2] + bz * X.kc;
  const int t1 = min(t0 + X.kc, L.hi[2] + 1);
  const int pbase = t0 - 2;  // first staged plane
  const uint32_t xtx = st.stall ? kStallBytes : 0u;
  const long long wlim = st.stall ? kStallLimit : kWaitLimit;

  // node role of this thread, a constant of the instantiation: 0 tile node,
  // 2 j-halo node (rows -1, TJ), 1 i-halo node (columns -1, TI)
  constexpr int role = ROLE;
  int nx, ny;
  if constexpr (ROLE == 0) {
    if (ROWS4) {  // warp w: rows (w & 3) + 8 (w >> 2) and 4 below it
      const int w = tid >> 5, l = tid & 31;
      nx = l & 15;
      ny = (w & 3) + 8 * (w >> 2) + 4 * (l >> 4);
    } else {
      nx = tid % TI;
      ny = tid / TI;
    }
  } else if constexpr (ROLE == 2) {
    const int h = tid - NTILE;
    nx = h % TI;
    ny = (h / TI) ? TJ : -1;
  } else {
    const int h = tid - NTILE - NJH;
    if (ROWS4) {  // both halo columns of four rows per quarter-warp: 2-way, not 4-way, bank conflicts
      ny = h >> 1;
      nx = (h & 1) ? TI : -1;
    } else {
      ny = h % TJ;
      nx = (h / TJ) ? TI : -1;
    }
  }
  const int gi = i0 + nx, gj = j0 + ny;
  const bool own = role == 0 && gi >= L.lo[0] && gi <= L.hi[0] && gj >= L.lo[1] && gj <= L.hi[1];

  // (re)initialise the barriers; every copy of the previous item has been
  // waited for, and every thread is past its last wait
  __syncthreads();
  if (tid == 0) {
    for (int b = 0; b < NBAR; ++b) {
      if (!first) mbar_inval(&sm.bar[b]);
      mbar_init(&sm.bar[b], 1);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // generic-proxy writes to the buffers the prologue stages into, then the barrier
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();

  // parities: the raw buffer takes plane t0-2, then t0+2, t0+3, ...; the
  // metric buffer planes t0-1, t0, ...
  auto raw_parity = [&](int p) { return (uint32_t)((p - t0 - 1) & 1); };
  auto met_parity = [&](int p) { return (uint32_t)((p - t0 + 1) & 1); };
  // thread 0's record of copies in flight: bit b of pend = barrier b has an
  // unwaited copy, bit b of ppar = the parity of that copy's phase
  uint32_t pend = 0, ppar = 0;
  auto issue_raw = [&](int p, int b, float* dst, uint32_t parity) {
    if (tid == 0) {
      pend |= 1u << b;
      ppar = (ppar & ~(1u << b)) | (parity << b);
      fence_async_shared();
      mbar_expect_tx(&sm.bar[b], RAW_TX + xtx);
      tma_load_4d(dst, &X.tmQ[st.qin], &sm.bar[b], i0, j0, p + NG, 0);
    }
  };
  auto issue_met = [&](int p) {
    if (tid == 0) {
      pend |= 1u << B_MET;
      ppar = (ppar & ~(1u << B_MET)) | ((uint32_t)((p - t0 + 1) & 1) << B_MET);
      fence_async_shared();
      mbar_expect_tx(&sm.bar[B_MET], MET_TX + xtx);
      tma_load_4d(sm.met, &X.tmMv, &sm.bar[B_MET], i0, j0 + 1, p + NG, 0);
    }
  };
  bool ok = true;
  auto wait = [&](int b, uint32_t parity, int p) {
    const bool r = wait_v(&sm.bar[b], parity, wlim);
    if (tid == 0) {
      if (r) pend &= ~(1u << b);
      else if (atomicCAS(X.err, 0, 1) == 0) {
        int* info = X.err + 1;
        info[0] = b; info[1] = (int)parity; info[2] = p; info[3] = bx; info[4] = by; info[5] = bz; info[6] = st.qin;
      }
    }
    ok = ok && r;
  };
  // ring slots of plane p: conserved (p - pbase) mod 4, primitive mod 3
  auto slot = [&](int p) { return ((p - pbase) & (NSQ - 1)) * RPL; };
  auto pslot = [&](int p) { return ((p - pbase) % NSP) * RPL; };

  // convert staged plane p (planar, in src) into the ring records: the
  // conserved record (CQ) and / or the primitive record (CP)
  auto convert_parts = [&](const float* src, int p, bool CQ, bool CP) {
    float4* qv = sm.QV + slot(p);
    float* qe = sm.QE + slot(p);
    float4* pv = sm.PV + pslot(p);
    float* pp = sm.PP + pslot(p);
    // halo threads (lighter in the node pass) take three elements each, tile
    // threads one or none
    const int e0 = tid < NTILE ? NCH + tid : tid - NTILE;
    const int e1 = tid < NTILE ? PL : NCH, es = tid < NTILE ? NTILE : NJH + NIH;
    for (int e = e0; e < e1; e += es) {
      const float q0 = src[e], q1 = src[PL + e], q2 = src[2 * PL + e], q3 = src[3 * PL + e], q4 = src[4 * PL + e];
      const float ri = Fn<float>::rcp(q0);
      const float u = q1 * ri, v = q2 * ri, w = q3 * ri;
      const float pr = c.gm1 * (q4 - 0.5f * q0 * (u * u + v * v + w * w));
      const int r = e + (RR - RW) * (e / RW);  // ring row (padded when RR > RW)
      if (CQ) {
        qv[r] = make_float4(q0, q1, q2, q3);
        qe[r] = q4;
      }
      if (CP) {
        pv[r] = make_float4(u, v, w, c.gamma * pr * ri);
        pp[r] = pr;
      }
    }
  };
  auto convert = [&](const float* src, int p) { convert_parts(src, p, true, true); };

  // node pass for plane kk: i/j node data to shared memory (for the
  // neighbours' faces) and in registers (for this thread's own faces), k data
  // in registers
  auto node_pass = [&](int kk, Own& w, float G3[5], float& lt3, float& nu3, float& Jn) {
    const int sM = pslot(kk - 1), sC = pslot(kk), sP = pslot(kk + 1), qC = slot(kk);
    float G[3][5], lt[3], nu[3];
    if (role == 0) {
      node_v<0, MD>(sm.PV, sm.PP, sm.QV, sm.QE, sm.met, sM, sC, sP, qC, nx, ny, c, G, lt, nu, Jn);
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        w.Gi[v] = G[0][v];
        w.Gj[v] = G[1][v];
        G3[v] = G[2][v];
      }
      w.Li = make_float2(lt[0], nu[0]);
      w.Lj = make_float2(lt[1], nu[1]);
      st5(sm.Gi4, sm.Gi1, ny * GIW + nx + 1, w.Gi);
      st5j(sm.Gj4, sm.Gj1, ny + 1, nx, w.Gj);
      sm.Li[ny * GIW + nx + 1] = w.Li;
      sm.Lj[(ny + 1) * TI + nx] = w.Lj;
      lt3 = lt[2];
      nu3 = nu[2];
    } else if (role == 1) {
      float Jh;
      node_v<1, MD>(sm.PV, sm.PP, sm.QV, sm.QE, sm.met, sM, sC, sP, qC, nx, ny, c, G, lt, nu, Jh);
#pragma unroll
      for (int v = 0; v < 5; ++v) { w.Gi[v] = G[0][v]; w.Gj[v] = 0.f; }
      w.Li = make_float2(lt[0], nu[0]);
      w.Lj = make_float2(0.f, 0.f);
      st5(sm.Gi4, sm.Gi1, ny * GIW + nx + 1, w.Gi);
      sm.Li[ny * GIW + nx + 1] = w.Li;
    } else {
      float Jh;
      node_v<2, MD>(sm.PV, sm.PP, sm.QV, sm.QE, sm.met, sM, sC, sP, qC, nx, ny, c, G, lt, nu, Jh);
#pragma unroll
      for (int v = 0; v < 5; ++v) { w.Gj[v] = G[1][v]; w.Gi[v] = 0.f; }
      w.Lj = make_float2(lt[1], nu[1]);
      w.Li = make_float2(0.f, 0.f);
      st5j(sm.Gj4, sm.Gj1, ny + 1, nx, w.Gj);
      sm.Lj[(ny + 1) * TI + nx] = w.Lj;
    }
  };

  // k data of plane kk only (tile threads), nothing written to shared memory
  auto node_pass_k = [&](int kk, float G3[5], float& lt3, float& nu3, float& Jn) {
    if (role != 0) return;
    float G[3][5], lt[3], nu[3];
    node_v<3, MD>(sm.PV, sm.PP, sm.QV, sm.QE, sm.met, pslot(kk - 1), pslot(kk), pslot(kk + 1), slot(kk), nx, ny, c, G,
              lt, nu, Jn);
#pragma unroll
    for (int v = 0; v < 5; ++v) G3[v] = G[2][v];
    lt3 = lt[2];
    nu3 = nu[2];
  };

  // face fluxes of plane kk on the low side of this thread's node: i face
  // between nx-1 and nx (tile nodes and the i-halo column TI), j face between
  // ny-1 and ny (tile nodes and the j-halo row TJ).  The node's own G, (lt, nu)
  // and conserved record come from registers; qo returns the record.
  const bool do_i = role == 0 || (role == 1 && nx == TI);
  const bool do_j = role == 0 || (role == 2 && ny == TJ);
  const int oo = (ny + 2) * RR + nx + 2;  // this thread's node in a ring plane
  auto face_pass = [&](int kk, const Own& w, float hi[5], float hj[5], float qo[5]) {
    const float4* qv = sm.QV + slot(kk);
    const float* qe = sm.QE + slot(kk);
    if (do_i || do_j) ld5(qv, qe, oo, qo);
    if (do_i) {
      float Ga[5], q0[5], q1[5], q3[5];
      ld5(sm.Gi4, sm.Gi1, ny * GIW + nx, Ga);
      ld5(qv, qe, oo - 2, q0);
      ld5(qv, qe, oo - 1, q1);
      ld5(qv, qe, oo + 1, q3);
      face_v(c, sm.Li[ny * GIW + nx], w.Li, Ga, w.Gi, q0, q1, qo, q3, hi);
      st5(sm.Hi4, sm.Hi1, ny * HIW + nx, hi);
    }
    if (do_j) {
      float Ga[5], q0[5], q1[5], q3[5];
      ld5j(sm.Gj4, sm.Gj1, ny, nx, Ga);
      ld5(qv, qe, oo - 2 * RR, q0);
      ld5(qv, qe, oo - RR, q1);
      ld5(qv, qe, oo + RR, q3);
      face_v(c, sm.Lj[ny * TI + nx], w.Lj, Ga, w.Gj, q0, q1, qo, q3, hj);
      st5j(sm.Hj4, sm.Hj1, ny, nx, hj);
    }
  };

  // i/j residual of this thread's tile node from the four face fluxes
  // around it (keeping the node's own faces in registers from the face
  // phase through the next node pass would exceed the register budget)
  auto rij = [&](float R[5]) {
    float a[5], b[5], d[5], e[5];
    ld5(sm.Hi4, sm.Hi1, ny * HIW + nx + 1, a);
    ld5(sm.Hi4, sm.Hi1, ny * HIW + nx, d);
    ld5j(sm.Hj4, sm.Hj1, ny + 1, nx, b);
    ld5j(sm.Hj4, sm.Hj1, ny, nx, e);
#pragma unroll
    for (int v = 0; v < 5; ++v) R[v] = (a[v] - d[v]) + (b[v] - e[v]);
  };

  // k face flux between planes ka and ka+1 of this thread's column; q1 is
  // the conserved record of plane ka+1 (already in registers)
  auto kface = [&](int ka, const float Ga[5], const float Gb[5], float lta, float ltb, float nua, float nub,
                   const float q1[5], float h[5]) {
    float qm[5], qa[5], qp[5];
    int s = slot(ka - 1);
    ld5(sm.QV + s, sm.QE + s, oo, qm);
    s = slot(ka);
    ld5(sm.QV + s, sm.QE + s, oo, qa);
    s = slot(ka + 2);
    ld5(sm.QV + s, sm.QE + s, oo, qp);
    face_v(c, make_float2(lta, nua), make_float2(ltb, nub), Ga, Gb, qm, qa, q1, qp, h);
  };

  const float adt = (float)(st.alpha * X.sc->dt);
  const long long npad = L.npad;
  float* const Qo = X.Q[st.qout];
  // Q^(0) of the plane being updated: for the first stage it is the stage
  // input, still in the conserved ring; otherwise TMA stages it one plane
  // ahead (tile rows, 36 columns from the aligned column i0-2)
  const bool q0_ring = st.qin == 0;
  const float* q0buf = reinterpret_cast<const float*>(smem + O_Q0);
  auto issue_q0 = [&](int p) {
    if (tid == 0 && !q0_ring) {
      pend |= 1u << B_Q0;
      ppar = (ppar & ~(1u << B_Q0)) | ((uint32_t)((p - t0) & 1) << B_Q0);
      fence_async_shared();
      mbar_expect_tx(&sm.bar[B_Q0], Q0_TX + xtx);
      tma_load_4d(smem + O_Q0, &X.tmQ0u, &sm.bar[B_Q0], i0, j0 + 2, p + NG, 0);
    }
  };
  long long n_t0 = own ? L.at(gi, gj, t0) : 0;  // this thread's node in plane t0
  float* scr[3] = {reinterpret_cast<float*>(smem + O_SCR), reinterpret_cast<float*>(smem + O_SCR + RAW_B),
                   reinterpret_cast<float*>(smem + O_SCR + 2 * RAW_B)};

  // ---- prologue: planes t0-2 .. t0+1 staged at once and converted
  issue_raw(t0 - 2, B_RAW, sm.raw, 0);
  issue_raw(t0 - 1, 1, scr[0], 0);
  issue_raw(t0, 2, scr[1], 0);
  issue_raw(t0 + 1, 3, scr[2], 0);
  issue_met(t0 - 1);
  wait(B_RAW, 0, t0 - 2);
  convert(sm.raw, t0 - 2);
  wait(1, 0, t0 - 1);
  convert(scr[0], t0 - 1);
  wait(2, 0, t0);
  convert(scr[1], t0);
  wait(3, 0, t0 + 1);
  // plane t0+1: conserved record now; its primitive slot still holds plane
  // t0-2, which the node pass of plane t0-1 reads
  convert_parts(scr[2], t0 + 1, true, false);
  if (__syncthreads_or(!ok)) goto fail;
  issue_raw(t0 + 2, B_RAW, sm.raw, raw_parity(t0 + 2));

  {
    float G3m[5], lt3m = 0.f, nu3m = 0.f, Jm = 0.f;
    float G3c[5], lt3c = 0.f, nu3c = 0.f, Jc = 0.f;
    float hprev[5];
    Own w;
    // node pass of plane t0-1 (its k data only), of plane t0, the k face
    // t0 - 1/2, the i/j faces of plane t0 and the conversion of plane t0+2
    wait(B_MET, met_parity(t0 - 1), t0 - 1);
    node_pass_k(t0 - 1, G3m, lt3m, nu3m, Jm);
    if (__syncthreads_or(!ok)) goto fail;
    issue_met(t0);
    convert_parts(scr[2], t0 + 1, false, true);  // scr[2] is overwritten by the node pass below
    if (__syncthreads_or(!ok)) goto fail;
    wait(B_MET, met_parity(t0), t0);
    node_pass(t0, w, G3c, lt3c, nu3c, Jc);
    if (role == 0) {
      float q1[5];
      const int s = slot(t0);
      ld5(sm.QV + s, sm.QE + s, oo, q1);
      kface(t0 - 1, G3m, G3c, lt3m, lt3c, nu3m, nu3c, q1, hprev);
    }
    if (__syncthreads_or(!ok)) goto fail;
    issue_met(t0 + 1);
    issue_q0(t0);
    {
      float hi[5], hj[5], qo[5];
      face_pass(t0, w, hi, hj, qo);
    }
    // ring slot of plane t0-2 is free: its last readers were the k face above
    wait(B_RAW, raw_parity(t0 + 2), t0 + 2);
    convert(sm.raw, t0 + 2);
    if (__syncthreads_or(!ok)) goto fail;
    if (t0 + 3 <= t1 + 1) issue_raw(t0 + 3, B_RAW, sm.raw, raw_parity(t0 + 3));

    // ---- march in k: iteration t writes plane t.  Phase 1: node pass of
    // plane t+1, k face t + 1/2, i/j residual of plane t (faces from phase 2
    // of the previous iteration) and the update of plane t.  Phase 2: i/j
    // faces of plane t+1 and the conversion of plane t+3 (into the ring slot
    // of plane t-1, whose last reader was the k face of phase 1).
    for (int t = t0; t < t1; ++t) {
      float G3n[5], lt3n = 0.f, nu3n = 0.f, Jn = 0.f;
      wait(B_MET, met_parity(t + 1), t + 1);
      node_pass(t + 1, w, G3n, lt3n, nu3n, Jn);
      if (!q0_ring) wait(B_Q0, (uint32_t)((t - t0) & 1), t);
      if (role == 0) {
        float q1[5], hk[5], R[5];
        const int s = slot(t + 1);
        ld5(sm.QV + s, sm.QE + s, oo, q1);
        kface(t, G3c, G3n, lt3c, lt3n, nu3c, nu3n, q1, hk);
        rij(R);
        if (own) {
          float q0[5];
          if (q0_ring) {
            const int s0 = slot(t);
            ld5(sm.QV + s0, sm.QE + s0, oo, q0);
          } else {
#pragma unroll
            for (int v = 0; v < 5; ++v) q0[v] = q0buf[v * UPL + ny * RW + nx + 2];
          }
          const long long n = n_t0 + (long long)(t - t0) * L.plane;
#pragma unroll
          for (int v = 0; v < 5; ++v) Qo[v * npad + n] = q0[v] - adt * Jc * (R[v] + (hk[v] - hprev[v]));
        }
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          G3c[v] = G3n[v];
          hprev[v] = hk[v];
        }
        lt3c = lt3n;
        nu3c = nu3n;
        Jc = Jn;
      }
      if (__syncthreads_or(!ok)) goto fail;
      if (t + 2 <= t1) issue_met(t + 2);
      if (t + 1 < t1) issue_q0(t + 1);
      if (t + 1 < t1) {
        float hi[5], hj[5], qo[5];
        face_pass(t + 1, w, hi, hj, qo);
      }
      if (t + 3 <= t1 + 1) {
        wait(B_RAW, raw_parity(t + 3), t + 3);
        convert(sm.raw, t + 3);
      }
      if (__syncthreads_or(!ok)) goto fail;
      if (t + 4 <= t1 + 1) issue_raw(t + 4, B_RAW, sm.raw, raw_parity(t + 4));
    }
  }
  return true;

fail:
  // let this item's copies in flight land before the shared memory is reused
  if (tid == 0) {
    atomicExch(X.err, 1);
    for (int b = 0; b < NBAR; ++b)
      if (pend & (1u << b)) {
        if (xtx) mbar_complete_tx(&sm.bar[b], xtx);
        mbar_wait_bounded(&sm.bar[b], (ppar >> b) & 1u);
      }
  }
  __syncthreads();
  return false;
}

template <int MD>
__global__ void __launch_bounds__(vr::NT, vr::MINB)
    k_stage_v(const __grid_constant__ StageCtx<float, float> X, const StageSel st) {
  extern __shared__ __align__(128) unsigned char smem[];
  switch (role_of(threadIdx.x)) {
    case 0: item_v<MD, 0>(X, st, blockIdx.x, blockIdx.y, blockIdx.z, smem, true); break;
    case 2: item_v<MD, 2>(X, st, blockIdx.x, blockIdx.y, blockIdx.z, smem, true); break;
    default: item_v<MD, 1>(X, st, blockIdx.x, blockIdx.y, blockIdx.z, smem, true); break;
  }
}

template <int MD>
__global__ void __launch_bounds__(vr::NT, vr::MINB)
    k_stage_v_batch(const StageCtx<float, float>* __restrict__ ctx, const int4* __restrict__ items, int nitems,
                    unsigned int* queue, const StageSel st) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ int next;
  bool first = true;
  for (;;) {
    if (threadIdx.x == 0) next = (int)atomicAdd(queue, 1u);
    __syncthreads();
    const int it = next;
    __syncthreads();
    if (it >= nitems) break;
    const int4 w = items[it];
    bool ok;
    switch (role_of(threadIdx.x)) {
      case 0: ok = item_v<MD, 0>(ctx[w.x], st, w.y, w.z, w.w, smem, first); break;
      case 2: ok = item_v<MD, 2>(ctx[w.x], st, w.y, w.z, w.w, smem, first); break;
      default: ok = item_v<MD, 1>(ctx[w.x], st, w.y, w.z, w.w, smem, first); break;
    }
    if (!ok) break;
    first = false;
  }
}

template <int MD>
cudaError_t configure_model() {
  cudaError_t e = cudaFuncSetAttribute(k_stage_v<MD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)vr::BYTES);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_stage_v_batch<MD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)vr::BYTES);
}

}  // namespace

cudaError_t VR_FN(stage_v_configure)() {
  cudaError_t e;
  if ((e = configure_model<kModelRuntime>()) != cudaSuccess) return e;
  if ((e = configure_model<kModelSmagorinsky>()) != cudaSuccess) return e;
  if ((e = configure_model<kModelVreman>()) != cudaSuccess) return e;
  return configure_model<kModelEuler>();
}

cudaError_t VR_FN(launch_stage_v)(const StageCtx<float, float>& X, const StageSel& st, cudaStream_t s) {
  const Layout& L = X.L;
  const int nz = L.hi[2] - L.lo[2] + 1;
  dim3 grid((L.hi[0] + vr::TI) / vr::TI, (L.hi[1] + vr::TJ) / vr::TJ, (nz + X.kc - 1) / X.kc);
  switch (flow_model(X.k)) {
    case kModelSmagorinsky: k_stage_v<kModelSmagorinsky><<<grid, vr::NT, vr::BYTES, s>>>(X, st); break;
    case kModelVreman: k_stage_v<kModelVreman><<<grid, vr::NT, vr::BYTES, s>>>(X, st); break;
    case kModelEuler: k_stage_v<kModelEuler><<<grid, vr::NT, vr::BYTES, s>>>(X, st); break;
    default: k_stage_v<kModelRuntime><<<grid, vr::NT, vr::BYTES, s>>>(X, st); break;
  }
  count_launches(1);
  return cudaGetLastError();
}

// model: the flow model every grid of the batch shares (kModelRuntime when
// they differ)
cudaError_t VR_FN(launch_stage_v_batch)(const void* ctx, const int4* items, int nitems, unsigned int* queue,
                                        const StageSel& st, int model, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(queue, 0, sizeof(unsigned int), s);
  if (e != cudaSuccess) return e;
  const int slots = device_sm_count() * vr::MINB;
  const int ctas = nitems < slots ? nitems : slots;
  const auto* X = (const StageCtx<float, float>*)ctx;
  switch (model) {
    case kModelSmagorinsky:
      k_stage_v_batch<kModelSmagorinsky><<<ctas, vr::NT, vr::BYTES, s>>>(X, items, nitems, queue, st);
      break;
    case kModelVreman: k_stage_v_batch<kModelVreman><<<ctas, vr::NT, vr::BYTES, s>>>(X, items, nitems, queue, st); break;
    case kModelEuler: k_stage_v_batch<kModelEuler><<<ctas, vr::NT, vr::BYTES, s>>>(X, items, nitems, queue, st); break;
    default: k_stage_v_batch<kModelRuntime><<<ctas, vr::NT, vr::BYTES, s>>>(X, items, nitems, queue, st); break;
  }
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace jz
