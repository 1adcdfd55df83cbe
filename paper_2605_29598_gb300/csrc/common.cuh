// Shared internals of libdgimex: context / mesh objects, 1D tables, error
// plumbing and the compile-time (dim, degree) dispatch.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/dgimex.h"
#include "df64.cuh"

namespace dg {

constexpr int MAX_N = 5;          // degree r <= 4
constexpr int MAX_NFP = 25;       // face points per face (r = 4, 3D)

__host__ __device__ constexpr int ipow(int b, int e) { return e == 0 ? 1 : b * ipow(b, e - 1); }

void set_error(const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what);

#define DG_CUDA(call)                                              \
  do {                                                             \
    cudaError_t e_ = (call);                                       \
    if (e_ != cudaSuccess) return ::dg::cuda_fail(e_, #call);      \
  } while (0)

#define DG_LAUNCH_CHECK(what)                                      \
  do {                                                             \
    cudaError_t e_ = cudaGetLastError();                           \
    if (e_ != cudaSuccess) return ::dg::cuda_fail(e_, what);       \
  } while (0)

// 1D tables of the Gauss-Legendre nodal basis on [0, 1], passed to kernels
// by value (they land in the constant bank).
template <typename T>
struct Tables {
  T D[MAX_N][MAX_N];         // D[k][j] = l_j'(xi_k)        (derivative at nodes)
  T L[2][MAX_N];             // L[s][j] = l_j(s)             (trace to face s)
  T P[2][MAX_N][MAX_N];      // P[b][q][j] = l_j((xi_q + b)/2)  (2:1 prolongation)
};

// A 1D matrix of the nodal change of basis between Gauss-Lobatto and
// Gauss-Legendre nodes (applied along every direction of a cell).
template <typename T>
struct Mat1D {
  T m[MAX_N][MAX_N];
};

struct HostTables {
  int n;
  double x[MAX_N], w[MAX_N];
  Tables<double> t;
  // Gauss-Lobatto nodes on [0, 1]; G[q][j] = l_j^GLL(x_q) (values at the
  // Gauss-Legendre points of the GLL nodal basis) and Gi[q][j] =
  // l_j^GL(xl_q) (its inverse: values at the GLL nodes of the GL basis)
  double xl[MAX_N];
  Mat1D<double> G, Gi;
};
void make_tables(int n, HostTables* out);   // Newton on Legendre P_n

template <typename T>
inline Tables<T> cast_tables(const Tables<double>& t) {
  Tables<T> o;
  for (int a = 0; a < MAX_N; ++a)
    for (int b = 0; b < MAX_N; ++b) {
      o.D[a][b] = (T)t.D[a][b];
      o.P[0][a][b] = (T)t.P[0][a][b];
      o.P[1][a][b] = (T)t.P[1][a][b];
    }
  for (int s = 0; s < 2; ++s)
    for (int b = 0; b < MAX_N; ++b) o.L[s][b] = (T)t.L[s][b];
  return o;
}

// Lazily grown device buffer owned by a mesh.
struct DBuf {
  void* p = nullptr;
  size_t bytes = 0;
  int ensure(size_t nbytes);
  void release();
  template <typename T> T* as() const { return static_cast<T*>(p); }
};

}  // namespace dg

namespace dg {

// Kernel classes counted (and optionally timed with CUDA events) between
// dg_profile_begin and dg_profile_end.
enum KernelId {
  K_TRACE = 0, K_FACE_EXPLICIT, K_HANG_GATHER, K_VOL_EXPLICIT, K_FACE_LAMBDA, K_FACE_GRAD,
  K_VOL_GRAD, K_FACE_DIV, K_VOL_DIV, K_USTAR, K_MULTIDOT, K_REDUCE, K_MULTIAXPY, K_VEC,
  K_STAGE, K_PICARD_NORMS, K_PRECOND, K_PRECOND_SETUP, K_COUNT   // K_PRECOND*: preconditioner solve / setup
};
extern const char* const kKernelNames[K_COUNT];

struct Profiler {
  bool on = false;
  uint32_t time_mask = 0;
  int64_t launches[K_COUNT] = {};
  std::vector<cudaEvent_t> pool;
  size_t used = 0;
  std::vector<int> pending_kid;      // kernel class of event pair k (events 2k, 2k+1)
  cudaEvent_t next_event();
  void reset();
  void release();
};

}  // namespace dg

struct dg_ctx {
  int device = 0;
};

struct dg_mesh {
  dg_ctx* ctx = nullptr;
  int dim = 0, degree = 0, n = 0, Np = 0, nfp = 0, nfaces = 0;
  int64_t E = 0, N = 0;
  int64_t S = 0;         // face slots = E * 2d * nfp
  int64_t nF = 0;        // unified face points
  int64_t nH = 0;        // hanging fine points
  int64_t nHC = 0;       // coarse hanging faces
  dg::HostTables tab;
  // geometry (device, FP64)
  double* verts = nullptr;   // E x 2^d x d
  double* K = nullptr;       // d*d x N : w det(J) (J^{-1})_{ab}
  double* invM = nullptr;    // N       : 1 / (w det J)
  double* fgeo = nullptr;    // (d+1) x nF : n dS (d comps), dS
  float* K32 = nullptr;      // FP32 copies for the mixed-precision path
  float* invM32 = nullptr;
  float* fgeo32 = nullptr;
  float* lv32 = nullptr;     // cell corners minus corner 0 (E x 2^d x d)
  float* tc32 = nullptr;     // terrain-following meshes: per cell 16 coefficients of
                             // the vertical row of J (see terrain_row in ops.cuh)
  // face-point topology (device, int32)
  int* fp_minus = nullptr;   // nF: minus slot
  int* fp_plus = nullptr;    // nF: plus slot, -1 wall, -2-hp hanging
  int* hp_cslot = nullptr;   // nH: coarse slot base (e_c*2d+f_c)*nfp
  int* hp_code = nullptr;    // nH: sub | (fine point index << 8)
  int* hc_slot = nullptr;    // nHC: coarse slot base
  int* cface = nullptr;      // E x 2d: neighbour across each cell face, -1 wall, -2 on a 2:1 face,
                             // -3 far field
  // far-field boundary (outer state = a given background state): per face
  // point its far-point index g (or -1; null without far-field faces), the
  // face points of the far list grouped by face type f = 0..2d-1
  // (far_fbeg[f] .. far_fbeg[f+1]), and the outer state's conserved traces
  // at the far points (5 x nFar, FP64 and FP32) once dg_mesh_set_far_state
  // has run
  int* fp_far = nullptr;
  int* far_p = nullptr;
  int64_t nFar = 0;
  int64_t far_fbeg[7] = {0, 0, 0, 0, 0, 0, 0};
  bool far_set = false;
  // workspace
  dg::DBuf trc, slot, hbuf, trh, pcoef, wv, gm_V, gm_work, red, st, fns, fs;
  dg::DBuf trh32, pcoef32, c32, ir32, irw;   // mixed precision: FP32 coefficients, IR vectors
  dg::DBuf irho, irho32;                      // 1/rho of the frozen stage density
  // fused face + cell kernels: implicit Rusanov coefficient per own face
  // slot (FP64, FP32) and outward n dS per own face slot (FP64: d x S)
  dg::DBuf pcs, pcs32, snS;
  int fused_stage[3] = {0, 1, 0};   // per precision (FP64, FP32, FP32 pairs): plus-side
                                    // values from the neighbour's node lines (1) or a
                                    // trace array (0); 2: one thread per x-line of a cell
                                    // (3D, degree 3; elsewhere as 1)
  // background of the perturbation-form explicit operator (mixed precision)
  dg::DBuf bg, bg32, bgF, bgtr, bgjump, pert32;
  // device-driven step (CUDA graph): solver state and fixed work vectors
  dg::DBuf gstate, gwork;
  // vertical-line preconditioner: chains of cells linked through conforming
  // bottom/top faces (device int32: cell above / below, -1 at a chain end;
  // first cell of each chain), FP32 block factors and work vectors
  int64_t n_vchains = 0;
  int* vl_above = nullptr;
  int* vl_below = nullptr;
  int* vl_heads = nullptr;
  dg::DBuf vl_slots, vl_fac, vl_scr, gm_pc;
  // cell-block preconditioner: per-slot face data, FP32 inverse cell blocks
  dg::DBuf cb_slots, cb_inv;
  int pc_kind = 0;   // DG_PRECOND_* of the factors last set up
  // Rayleigh damping layers: lambda (N) then q_bar (5 x N)
  dg::DBuf sponge;
  bool sponge_set = false;
  struct StepGraph* graph = nullptr;   // cached executable graph of imex_ark2_step
  bool bg_set = false;
  double bg_gamma = 0, bg_g = 0, bg_f = 0, bg_lmin = 0;
  const double* bg_fcell = nullptr;
  std::vector<double> host_h;
  dg::Profiler prof;
  // cells-per-block multiplier of the cell kernels, per class (FP64, FP32)
  int tile[dg::K_COUNT] = {1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1};
  int tile32[dg::K_COUNT] = {1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1};
  int tilep[dg::K_COUNT] = {1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1};   // FP32 pairs
  // every cell terrain-following: x depends on xi_1 only and y on xi_2 only
  // (rectangular footprints, any vertical map), so the metric terms
  // K_ab = w det(J) (J^-1)_ab vanish exactly for (a, b) = (1, y), (1, z),
  // (2, x), (2, z) (3D) or (1, z) (2D) and the cell kernels skip them
  bool terrain = false;
  // Gauss-Lobatto nodal basis (Section 3.1's S^{-1} W^{-1} S^{-T} inverse
  // mass): every nodal array at the ABI is in the GLL basis; the operators
  // run in the Gauss-Legendre basis of the same polynomials and the arrays
  // are converted per cell on the way in and out
  bool gll = false;
  dg::DBuf gl64, gl32, gldf;   // GL copies of coefficients (5N) and inputs (5N): FP64, FP32, pairs
  dg::DBuf far_q, far_q32, farw;   // outer traces (FP64, FP32); predictors with the outer data (4N)
  dg::DBuf far_qdf;                // outer traces as FP32 pairs (DG_PAIRS)
  // DG_PAIRS (FP64-class vmults on the FP32 pipe): pair copies of the
  // geometry (metric, 1/(w det J), face n dS and dS, per-slot normals), of the
  // frozen coefficients (5N + E) and their face data, and the vmult's x, y
  dg::DBuf Kdf, invMdf, fgeodf, snSdf, cdf, trhdf, pcoefdf, irhodf, pcsdf, irdf;
  int64_t workspace_bytes() const;
  // every workspace buffer, for accounting, release and graph capture checks
  static constexpr int kBufs = 54;
  void bufs(const dg::DBuf** out) const {
    const dg::DBuf* b[kBufs] = {&trc, &slot, &hbuf, &trh, &pcoef, &wv, &gm_V, &gm_work, &red, &st,
                                &fns, &fs, &trh32, &pcoef32, &c32, &ir32, &irw, &irho, &irho32,
                                &bg, &bg32, &bgF, &bgtr, &bgjump, &pert32, &gstate, &gwork,
                                &vl_slots, &vl_fac, &vl_scr, &gm_pc, &sponge,
                                &cb_slots, &cb_inv, &pcs, &pcs32, &snS, &gl64, &gl32, &far_q, &far_q32,
                                &farw, &Kdf, &invMdf, &fgeodf, &snSdf, &cdf, &trhdf, &pcoefdf, &irhodf,
                                &pcsdf, &irdf, &far_qdf, &gldf};
    for (int i = 0; i < kBufs; ++i) out[i] = b[i];
  }
};

namespace dg {

// releases the cached step graph of a mesh (defined with the graph code)
void graph_release(dg_mesh* m);
// outward n dS of every face slot (d x S, own cell), mesh.cu
int slot_normals(const dg_mesh* m, double* out, cudaStream_t st);

}  // namespace dg

struct MultiGraph;   // several meshes' steps captured as one graph

namespace dg {

void multi_graph_release(MultiGraph* g);
int multi_step_graph(int ng, dg_mesh* const* meshes, const dg_phys* phs, double* const* qs, const double* dts,
                     const dg_step_opts* o, dg_step_info* infos, MultiGraph** cache, cudaStream_t st);

// Arguments shared by the face kernels.
struct FaceTopo {
  const int* fp_minus;
  const int* fp_plus;
  const double* fgeo;
  const float* fgeo32;
  const int* hp_cslot;
  const int* hp_code;
  const int* hc_slot;
  int64_t nF, nH, nHC, S;
  int64_t p0;   // first face point a face kernel handles (0: all of them)
  // far-field points among the boundary ones (code -1): index g into the
  // outer traces (5 x nFar), or -1 for a wall; fp_far null: walls only
  const int* fp_far;
  const double* far_q;
  const float* far_q32;
  int64_t nFar;
  const df64* fgeodf;   // face geometry as FP32 pairs (DG_PAIRS), or null
  const df64* far_qdf;  // outer traces as FP32 pairs (DG_PAIRS), or null
};

inline FaceTopo topo(const dg_mesh* m) {
  return FaceTopo{m->fp_minus, m->fp_plus, m->fgeo, m->fgeo32, m->hp_cslot, m->hp_code,
                  m->hc_slot, m->nF, m->nH, m->nHC, m->S, 0,
                  m->nFar > 0 ? m->fp_far : nullptr, m->far_q.as<double>(), m->far_q32.as<float>(), m->nFar,
                  m->fgeodf.as<df64>(), m->far_qdf.as<df64>()};
}

// the face points of the 2:1 faces only (the last nH of the unified list)
inline FaceTopo topo_hanging(const dg_mesh* m) {
  FaceTopo ft = topo(m);
  ft.p0 = m->nF - m->nH;
  return ft;
}

// Counts a launch of class `kid` and brackets it with CUDA events when that
// class is being timed.
struct ProfScope {
  Profiler* p;
  int kid;
  cudaStream_t st;
  cudaEvent_t stop = nullptr;
  ProfScope(dg_mesh* m, int k, cudaStream_t s) : p(&m->prof), kid(k), st(s) {
    if (!p->on) return;
    p->launches[kid]++;
    if (p->time_mask & (1u << kid)) {
      cudaEvent_t start = p->next_event();
      stop = p->next_event();
      if (start && stop) {
        cudaEventRecord(start, st);
        p->pending_kid.push_back(kid);
      } else {
        stop = nullptr;
      }
    }
  }
  ~ProfScope() {
    if (stop) cudaEventRecord(stop, st);
  }
};

#define DG_RUN(m, kid, st, ...)                      \
  do {                                               \
    ::dg::ProfScope prof_scope_((m), (kid), (st));   \
    __VA_ARGS__;                                     \
  } while (0)

inline unsigned grid_for(int64_t n, int threads) {
  int64_t g = (n + threads - 1) / threads;
  return (unsigned)(g < 1 ? 1 : g);
}

}  // namespace dg
