// Per-(T, DIM, N) operator engine and the runtime (dim, degree) dispatch.
#pragma once

#include "ops.cuh"

namespace dg {

template <typename T, int DIM, int N>
struct Engine {
  static int explicit_rates(dg_mesh* m, const PhysK& ph, const T* q, T* fns, T* fs, cudaStream_t st);
  static int prepare(dg_mesh* m, const ImplK& ph, const T* rho, const T* plag, const T* ulag, int penalty,
                     cudaStream_t st);
  static int vmult(dg_mesh* m, const ImplK& ph, const T* rho, const T* plag, int penalty, const T* x, T* y,
                   cudaStream_t st);
  static int schur_rhs(dg_mesh* m, const ImplK& ph, const T* rho, const T* plag, const T* ulag, const T* mhat,
                       const T* ehat, T* rhs, cudaStream_t st);
  static int recover(dg_mesh* m, const ImplK& ph, const T* rho, const T* ulag, const T* mhat, const T* p, T* u,
                     cudaStream_t st);
};

ImplK impl_consts(const dg_phys* ph, double a_dt);

// Per-precision views of the mesh geometry and of the per-Picard
// coefficient buffers (FP32 copies are made by ensure_fp32_geometry).
template <typename T> inline const T* met_K(const dg_mesh* m);
template <> inline const double* met_K<double>(const dg_mesh* m) { return m->K; }
template <> inline const float* met_K<float>(const dg_mesh* m) { return m->K32; }
template <> inline const df64* met_K<df64>(const dg_mesh* m) { return m->Kdf.as<df64>(); }
template <typename T> inline const T* met_invM(const dg_mesh* m);
template <> inline const double* met_invM<double>(const dg_mesh* m) { return m->invM; }
template <> inline const float* met_invM<float>(const dg_mesh* m) { return m->invM32; }
template <> inline const df64* met_invM<df64>(const dg_mesh* m) { return m->invMdf.as<df64>(); }
// per-precision coefficient buffers: FP64, FP32 and FP32 pairs each own one
template <typename T> inline DBuf& buf_trh(dg_mesh* m);
template <> inline DBuf& buf_trh<double>(dg_mesh* m) { return m->trh; }
template <> inline DBuf& buf_trh<float>(dg_mesh* m) { return m->trh32; }
template <> inline DBuf& buf_trh<df64>(dg_mesh* m) { return m->trhdf; }
template <typename T> inline DBuf& buf_pcoef(dg_mesh* m);
template <> inline DBuf& buf_pcoef<double>(dg_mesh* m) { return m->pcoef; }
template <> inline DBuf& buf_pcoef<float>(dg_mesh* m) { return m->pcoef32; }
template <> inline DBuf& buf_pcoef<df64>(dg_mesh* m) { return m->pcoefdf; }
template <typename T> inline DBuf& buf_irho(dg_mesh* m);
template <> inline DBuf& buf_irho<double>(dg_mesh* m) { return m->irho; }
template <> inline DBuf& buf_irho<float>(dg_mesh* m) { return m->irho32; }
template <> inline DBuf& buf_irho<df64>(dg_mesh* m) { return m->irhodf; }
int ensure_fp32_geometry(dg_mesh* m);

// Metric source of the implicit cell kernels: FP64 loads the stored
// metric; FP32 recomputes it from the cell corner offsets.
template <typename T>
inline CellGeo<T> cell_geo(const dg_mesh* m) {
  CellGeo<T> g;
  g.K = met_K<T>(m);
  g.invM = met_invM<T>(m);
  g.lv = nullptr;
  g.tc = nullptr;
  for (int k = 0; k < MAX_N; ++k) {
    g.x[k] = (T)m->tab.x[k];
    g.w[k] = (T)m->tab.w[k];
  }
  g.terrain = m->terrain ? 1 : 0;
  return g;
}
template <>
inline CellGeo<float> cell_geo<float>(const dg_mesh* m) {
  CellGeo<float> g;
  g.K = m->K32;
  g.invM = m->invM32;
  g.lv = m->lv32;
  g.tc = m->tc32;
  for (int k = 0; k < MAX_N; ++k) {
    g.x[k] = (float)m->tab.x[k];
    g.w[k] = (float)m->tab.w[k];
  }
  g.terrain = m->terrain ? 1 : 0;
  return g;
}
// Explicit operator in perturbation form about the mesh's background (FP32
// differences + FP64 background rates); requires m->bg_set.
int explicit_mixed(dg_mesh* m, const PhysK& ph, const double* q, double* fns, double* fs, cudaStream_t st);
// FP32 rates of q as increments about a reference state q0 whose FP64 rates
// are f0: increment_begin prepares the face data of q0 (once per q0)
int increment_begin(dg_mesh* m, double gamma, const double* q0, cudaStream_t st);
int explicit_increment(dg_mesh* m, const PhysK& ph, const double* q, const double* q0, const double* f0_ns,
                       const double* f0_s, double* fns, double* fs, cudaStream_t st);
// fns -= lambda (q - q_bar) when the mesh has damping layers (sponge.cu);
// with ref, fns -= lambda (q - ref): the damping increment for rates that
// were formed as increments about ref from rates that already hold the
// damping at ref
int sponge_rt(dg_mesh* m, const double* q, double* fns, cudaStream_t st, const double* ref = nullptr);
// Gauss-Lobatto meshes: out = G in (to_gl) or G^{-1} in per cell, nfld
// fields of N doubles (in == out allowed); gl_scratch: 5N doubles of FP64
// scratch after the GL copies of the frozen coefficients (null when the
// allocation fails)
int gl_basis(dg_mesh* m, const double* in, double* out, int nfld, bool to_gl, cudaStream_t st);
double* gl_scratch(dg_mesh* m);
// DG_PAIRS: pair copies of the geometry (made once per mesh), and FP64 <->
// pair conversions of n values
int ensure_pairs_geometry(dg_mesh* m, cudaStream_t st);
int to_pairs(dg_mesh* m, const double* a, df64* b, int64_t n, cudaStream_t st);
int from_pairs(dg_mesh* m, const df64* a, double* b, int64_t n, cudaStream_t st);
int schur_vmult_pairs(dg_mesh* m, const ImplK& k, const double* rho, const double* plag, const double* ulag,
                      int penalty, const double* x, double* y, cudaStream_t st);
// FP32 Schur vmult (coefficients and vectors cast from / to FP64)
int schur_vmult_mixed(dg_mesh* m, const ImplK& k, const double* rho, const double* plag, const double* ulag,
                      int penalty, const double* x, double* y, cudaStream_t st);

// Run the statement list with the tile multiplier M_ (cells per block =
// M_ x the base count) chosen for kernel class `kid` of the mesh.
template <typename T> inline int tile_of(const dg_mesh* m, int kid) {
  return std::is_same<T, float>::value ? m->tile32[kid]
                                       : (std::is_same<T, double>::value ? m->tile[kid] : m->tilep[kid]);
}
#define DG_TILE(m, kid, ...)                                         \
  switch (tile_of<T>((m), kid)) {                                    \
    case 2: { constexpr int M_ = 2; __VA_ARGS__; } break;            \
    case 4: { constexpr int M_ = 4; __VA_ARGS__; } break;            \
    default: { constexpr int M_ = 1; __VA_ARGS__; } break;           \
  }

// Run the statement list for the mesh's compile-time (dim, n): D_ and N_ are
// constexpr inside it.
#define DG_DISPATCH(m, ...)                                  \
  switch ((m)->dim * 10 + (m)->n) {                          \
    case 22: { constexpr int D_ = 2, N_ = 2; __VA_ARGS__; } break; \
    case 23: { constexpr int D_ = 2, N_ = 3; __VA_ARGS__; } break; \
    case 24: { constexpr int D_ = 2, N_ = 4; __VA_ARGS__; } break; \
    case 25: { constexpr int D_ = 2, N_ = 5; __VA_ARGS__; } break; \
    case 32: { constexpr int D_ = 3, N_ = 2; __VA_ARGS__; } break; \
    case 33: { constexpr int D_ = 3, N_ = 3; __VA_ARGS__; } break; \
    case 34: { constexpr int D_ = 3, N_ = 4; __VA_ARGS__; } break; \
    case 35: { constexpr int D_ = 3, N_ = 5; __VA_ARGS__; } break; \
    default: break;                                          \
  }

}  // namespace dg
