// jz_internal.h -- launchers shared between the translation units of the
// library (host-side declarations; not part of the public ABI).
#pragma once

#include <cstdint>
#include <vector>
#include <cuda.h>
#include <cuda_runtime.h>

#include "jz_common.cuh"

namespace jz {

// Everything a kernel launcher needs to know about one grid on the device.
struct GridDev {
  Layout L;
  int prec;            // JZ_P64, JZ_P32_M64, JZ_P32
  void* Q0;            // Q^n, then Q^(5) in place
  double* Q0d;         // JZ_P32_S64: the FP64 state Q^n at the updated nodes (else null)
  void* QA;            // Q^(1), Q^(3)
  void* QB;            // Q^(2), Q^(4)
  void* M;             // metrics: S^k_m at field 3k+m, J at field 9
  Coords C;            // coordinate tables
  Scalars* sc;         // device scalars
  double* partial;     // reduction partials: RED_BLOCKS * (DIAG_WORDS + 1) doubles
  double* inflow;      // axial inflow velocity at the x- face nodes, [k][j] (set by state_init)
  double* axis;        // centreline values of a cylindrical grid, [5][ni] FP64 (set per boundary pass)
  FlowC F;
  int kc;              // planes per CTA chunk of the stage kernel
  int goff[3], gn[3];  // global index of local node 0 and global node counts (blocks; else 0 and n)
  int variant;         // stage kernel of P32: 0 scalar records, 2 vector records
  int vti, vtj;        // tile shape of the vector-record kernel (32 x 16, 16 x 32 or 16 x 16)
  int stall_test;      // test only: the stage kernels' copies wait for bytes that nothing delivers
  int step_diag;       // each step's time-step reduction also forms the diagnostics of the state it reads
  CUtensorMap tmQ[3];  // TMA maps of Q0, QA, QB (stage kernel tile box)
  CUtensorMap tmM;     // TMA map of the metric fields
  CUtensorMap tmMv;    // the same fields, box of the tile plus a one-node halo (P32)
  CUtensorMap tmQ0u;   // Q0, box of the tile rows only (P32)
};

// Interior-vs-shell enumeration: every padded node outside the box [a, b].
struct Shell {
  int a[3], b[3], E[3];
  long long cz, cy, cx;  // node counts of the z, y and x slabs
  __host__ __device__ long long total() const { return cz + cy + cx; }
};
Shell make_shell(const Layout& L, const int a[3], const int b[3]);

struct TabParams {
  int n[3], per[3], pn[3];
  int cyl;
  int off[3], gn[3];  // global index of local node 0, global node counts (a block of a larger grid)
  double lo[3], hi[3];
  double cluster_r, stretch_c, stretch_w, amp;
  int m[9];
  double th[9];
};

// jz_api.cu: set the calling thread's jz_last_error message; returns code
int record_error(int code, const char* msg);

// jz_grid.cu
cudaError_t launch_tables(const TabParams& p, double* tables, cudaStream_t s);
cudaError_t launch_metrics(const GridDev& g, cudaStream_t s);
cudaError_t launch_init(const GridDev& g, uint64_t seed, cudaStream_t s);
cudaError_t launch_bc(const GridDev& g, void* Q, cudaStream_t s, bool full = false);
cudaError_t launch_unpack(const GridDev& g, const double* dense, cudaStream_t s);
cudaError_t launch_pack(const GridDev& g, double* dense, cudaStream_t s);
// one metric field (S^k_m at 3k+m, J at 9) of the grid's own nodes, widened to FP64
cudaError_t launch_pack_metric(const GridDev& g, int f, double* dense, cudaStream_t s);

// batched boundary fill over a device table of per-grid contexts
size_t bc_ctx_bytes();
void bc_ctx_fill(void* host_dst, const GridDev& g);
// batched boundary pass: work items (grid, slab, first node, end node) of at
// most BC_ITEM_NODES nodes (one 256-thread block each)
constexpr int BC_ITEM_NODES = 1024;
void bc_fill_items(const GridDev& g, int grid, std::vector<int4>& out);
cudaError_t launch_bc_batch(int prec, const void* ctx, int n, const int4* items, int nitems, int which, bool cyl,
                            cudaStream_t s);

// halo exchange between blocks of one grid: one entry per (block, exchange face)
struct XEntry {
  void* dq[3];                       // Q0, QA, QB of the block whose ghosts are filled
  void* sq[3];                       // Q0, QA, QB of the neighbouring block
  long long dpitch, dplane, dnpad;   // strides (elements) of the two layouts
  long long spitch, splane, snpad;
  int d;                             // direction of the face normal
  int dfirst, sfirst;                // first local index along d of the ghost layers / the copied layers
  int ea, eb;                        // padded node counts of the other two directions (i, j, k order)
};
cudaError_t launch_exchange(int prec, const void* entries, int begin, int count, int blocks, int which,
                            cudaStream_t s);
// two node layers [first, first + 1] along d (padded extents of the other
// directions) of state Q to / from a dense buffer (pack: state -> buffer)
cudaError_t launch_halo(const GridDev& g, void* Q, void* buf, int d, int first, bool pack, cudaStream_t s);
// a block's stable-step rate into sc->rate (no time step taken), and the
// time step from a rate already combined over the grid's blocks
cudaError_t launch_rate(const GridDev& g, cudaStream_t s);
cudaError_t launch_advance_from_rate(const GridDev& g, double cfl, cudaStream_t s);

// jz_stats.cu: time statistics of the axial velocity
cudaError_t launch_stats_sample(const GridDev& g, double* su, double* su2, cudaStream_t s);
cudaError_t launch_stats_plane_yz(const GridDev& g, int i, double* yz, cudaStream_t s);
cudaError_t launch_stats_axis_x(const GridDev& g, int jc, int kc, double* x, cudaStream_t s);

// jz_reduce.cu
cudaError_t launch_timestep(const GridDev& g, double cfl, double dt_fixed, cudaStream_t s);
cudaError_t launch_diagnostics(const GridDev& g, cudaStream_t s);
size_t rate_ctx_bytes();
void rate_ctx_fill(void* host_dst, const GridDev& g);
// coupled: the grids are blocks of one grid and share its time step
cudaError_t launch_timestep_batch(int prec, const void* ctx, int n, double cfl, bool coupled, cudaStream_t s);

// jz_stage.cu
struct StageTiling { int ti, tj; };
StageTiling stage_tiling(int prec);
// the tile of the kernel a grid runs: its chosen shape for the FP32
// vector-record kernel, else the fixed tile of its precision mode
inline StageTiling grid_tiling(const GridDev& g) {
  return (g.prec == JZ_P32 && g.variant == 2) ? StageTiling{g.vti, g.vtj} : stage_tiling(g.prec);
}
int stage_ctas_per_sm(int prec);
// resident CTAs per SM of the stage kernel a grid runs
int grid_ctas_per_sm(const GridDev& g);
// streaming multiprocessors of the current device (queried once per device)
int device_sm_count();
// qsel / qout select the input state Q^(l-1) and the output Q^(l): 0 = Q0, 1 = QA, 2 = QB
cudaError_t launch_stage(const GridDev& g, int stage, int qsel, int qout, cudaStream_t s);
// batched stage: a device table of per-grid stage contexts and work items
size_t stage_ctx_bytes(int prec);
void stage_ctx_fill(void* host_dst, const GridDev& g);
// the flow model a grid's FP32 vector-record stage kernel is compiled for
// (the runtime model when none of the constant-flag builds matches)
int stage_model(const GridDev& g);
// model: the stage_model shared by every grid of the batch, else the runtime model
cudaError_t launch_stage_batch(int prec, int variant, StageTiling tile, const void* ctx, const int4* items,
                               int nitems, unsigned int* queue, int stage, int qsel, int qout, int model,
                               cudaStream_t s);
cudaError_t stage_configure();  // one-time kernel attributes (dynamic shared memory)

}  // namespace jz
