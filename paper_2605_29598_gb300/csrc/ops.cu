// Launch sequences of the explicit operator, the Schur-complement vmult,
// the Schur right-hand side and the velocity recovery, plus their C entry
// points.
#include "engine.cuh"
#include "fused.cuh"
#include "lines.cuh"

namespace dg {

// Outward n dS per own face slot for the fused kernels: FP64 loads them
// (computed once per mesh, exact negatives across every conforming face);
// FP32 recomputes them from the cell corner offsets (null here).
template <typename T> static int fused_normals(dg_mesh* m, cudaStream_t st, const T** out);
template <>
int fused_normals<float>(dg_mesh* m, cudaStream_t, const float** out) {
  if (!m->lv32) {
    set_error("fused FP32 kernels: FP32 geometry not prepared");
    return DG_ERR_ARG;
  }
  *out = nullptr;
  return DG_OK;
}
template <>
int fused_normals<df64>(dg_mesh* m, cudaStream_t, const df64** out) {
  if (!m->snSdf.p) {
    set_error("DG_PAIRS kernels: pair geometry not prepared");
    return DG_ERR_ARG;
  }
  *out = m->snSdf.as<df64>();
  return DG_OK;
}
template <>
int fused_normals<double>(dg_mesh* m, cudaStream_t st, const double** out) {
  if (!m->snS.p) {
    int rc;
    if ((rc = m->snS.ensure(sizeof(double) * m->dim * (m->S > 0 ? m->S : 1))) != DG_OK) return rc;
    if ((rc = slot_normals(m, m->snS.as<double>(), st)) != DG_OK) return rc;
  }
  *out = m->snS.as<double>();
  return DG_OK;
}

template <typename T> inline DBuf& buf_pcs(dg_mesh* m);
template <> inline DBuf& buf_pcs<double>(dg_mesh* m) { return m->pcs; }
template <> inline DBuf& buf_pcs<float>(dg_mesh* m) { return m->pcs32; }
template <> inline DBuf& buf_pcs<df64>(dg_mesh* m) { return m->pcsdf; }

// Gauss-Lobatto meshes.  The operators run in the Gauss-Legendre nodal
// basis of the same polynomials, with the same quadrature: a GLL nodal
// vector v has GL nodal values G v (G = interpolation of the GLL basis to
// the GL points, per direction), nodal rates and Schur vectors transform
// the same way, and the GLL inverse mass S^{-1} W^{-1} S^{-T} of Section 3.1
// becomes G^{-1} (GL inverse mass) on the way out.  Buffer layout per
// precision: [0, 5N) GL copies of rho, p_lag, u_lag (from prepare), [5N,
// 10N) GL copies of the other inputs of one call.
template <typename T> inline DBuf& buf_gl(dg_mesh* m) {
  return std::is_same<T, float>::value ? m->gl32 : (std::is_same<T, double>::value ? m->gl64 : m->gldf);
}
template <typename T>
inline Mat1D<T> cast_mat(const Mat1D<double>& a) {
  Mat1D<T> o;
  for (int i = 0; i < MAX_N; ++i)
    for (int j = 0; j < MAX_N; ++j) o.m[i][j] = (T)a.m[i][j];
  return o;
}
// out = G in (to_gl) or G^{-1} in, nfld fields of N values; in == out allowed
template <typename T, int DIM, int N>
static void gl_convert(dg_mesh* m, const T* in, T* out, int nfld, bool to_gl, cudaStream_t st) {
  using CS = CellShape<DIM, N>;
  DG_RUN(m, K_VEC, st, k_basis<T, DIM, N><<<grid_for(m->E, CS::EPB), CS::THREADS, 0, st>>>(
                           in, out, nfld, m->E, cast_mat<T>(to_gl ? m->tab.G : m->tab.Gi)));
}
template <typename T>
static int gl_buffers(dg_mesh* m) {
  return buf_gl<T>(m).ensure(sizeof(T) * 10 * (size_t)m->N);
}

// far-field faces need their outer state before any operator runs
static int far_ready(const dg_mesh* m) {
  if (m->nFar > 0 && !m->far_set) {
    set_error("the mesh has far-field faces: set their outer state with dg_mesh_set_far_state first");
    return DG_ERR_ARG;
  }
  return DG_OK;
}

// Stage predictors with the far-field outer data moved to them (see
// k_far_affine): copies of m_hat (and e_hat, when given) in the mesh's farw
// buffer, corrected face type by face type; the pointers are redirected.
template <typename T, int DIM, int N>
static int far_predictors(dg_mesh* m, const ImplK& ph, const T*& mhat, const T*& ehat, cudaStream_t st) {
  if (m->nFar == 0) return DG_OK;
  int rc;
  if ((rc = m->farw.ensure(sizeof(T) * 4 * (size_t)m->N)) != DG_OK) return rc;
  T* w = m->farw.template as<T>();
  DG_CUDA(cudaMemcpyAsync(w, mhat, sizeof(T) * 3 * m->N, cudaMemcpyDeviceToDevice, st));
  if (ehat) DG_CUDA(cudaMemcpyAsync(w + 3 * m->N, ehat, sizeof(T) * m->N, cudaMemcpyDeviceToDevice, st));
  Tables<T> tb = cast_tables<T>(m->tab.t);
  const FaceTopo ft = topo(m);
  const T* pcoef = ph.penalty ? buf_pcoef<T>(m).template as<T>() : nullptr;
  for (int f = 0; f < 2 * DIM; ++f) {
    const int64_t g0 = m->far_fbeg[f], g1 = m->far_fbeg[f + 1];
    if (g1 > g0)
      DG_RUN(m, K_USTAR, st, k_far_affine<T, DIM, N><<<grid_for(g1 - g0, 128), 128, 0, st>>>(
                                 ft, m->far_p, g0, g1, f, met_invM<T>(m), pcoef, ph, tb, w,
                                 ehat ? w + 3 * m->N : nullptr, m->N));
  }
  mhat = w;
  if (ehat) ehat = w + 3 * m->N;
  return DG_OK;
}

// outer conserved traces at the far points from the trace array
__global__ void k_far_gather(const int* __restrict__ far_p, const int* __restrict__ fp_minus,
                             const double* __restrict__ trc, int64_t S, int64_t nFar, double* __restrict__ fq,
                             float* __restrict__ fq32, df64* __restrict__ fqdf) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= nFar) return;
  const int sm = fp_minus[far_p[g]];
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const double v = trc[k * S + sm];
    fq[k * nFar + g] = v;
    fq32[k * nFar + g] = (float)v;
    fqdf[k * nFar + g] = df64(v);
  }
}

template <int DIM, int N>
static int set_far_state(dg_mesh* m, const double* q, cudaStream_t st) {
  int rc;
  if ((rc = m->trc.ensure(sizeof(double) * 5 * m->S)) != DG_OK) return rc;
  if ((rc = m->far_q.ensure(sizeof(double) * 5 * m->nFar)) != DG_OK) return rc;
  if ((rc = m->far_q32.ensure(sizeof(float) * 5 * m->nFar)) != DG_OK) return rc;
  if ((rc = m->far_qdf.ensure(sizeof(df64) * 5 * m->nFar)) != DG_OK) return rc;
  if (m->gll) {
    if ((rc = gl_buffers<double>(m)) != DG_OK) return rc;
    double* qg = m->gl64.as<double>() + 5 * m->N;
    gl_convert<double, DIM, N>(m, q, qg, 5, true, st);
    q = qg;
  }
  Tables<double> tb = cast_tables<double>(m->tab.t);
  Fields<double> in;
  for (int k = 0; k < 5; ++k) {
    in.f[k] = q + k * m->N;
    in.scale[k] = 1;
  }
  k_trace<double, DIM, N, 5><<<trace_grid<DIM, N>(m->E), TraceShape<DIM, N>::THREADS, 0, st>>>(
      in, m->E, m->N, m->trc.as<double>(), m->S, tb);
  k_far_gather<<<grid_for(m->nFar, 128), 128, 0, st>>>(m->far_p, m->fp_minus, m->trc.as<double>(), m->S, m->nFar,
                                                         m->far_q.as<double>(), m->far_q32.as<float>(),
                                                         m->far_qdf.as<df64>());
  DG_LAUNCH_CHECK("far-field outer state");
  m->far_set = true;
  return DG_OK;
}
template <typename T> inline int fused_sched(const dg_mesh* m) {
  return m->fused_stage[std::is_same<T, double>::value ? 0 : (std::is_same<T, float>::value ? 1 : 2)];
}
template <typename T> inline bool fused_stage(const dg_mesh* m) { return fused_sched<T>(m) != 0; }
inline bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

template <typename T, int DIM, int N>
int Engine<T, DIM, N>::explicit_rates(dg_mesh* m, const PhysK& ph, const T* q, T* fns, T* fs,
                                      cudaStream_t st) {
  using CS = CellShape<DIM, N>;
  int rc;
  if ((rc = far_ready(m)) != DG_OK) return rc;
  if ((rc = m->trc.ensure(sizeof(T) * 5 * m->S)) != DG_OK) return rc;
  if ((rc = m->slot.ensure(sizeof(T) * 9 * m->S)) != DG_OK) return rc;
  if ((rc = m->hbuf.ensure(sizeof(T) * 9 * (m->nH > 0 ? m->nH : 1))) != DG_OK) return rc;
  if (m->gll) {
    if ((rc = gl_buffers<T>(m)) != DG_OK) return rc;
    T* qg = buf_gl<T>(m).template as<T>() + 5 * m->N;
    gl_convert<T, DIM, N>(m, q, qg, 5, true, st);
    q = qg;
  }
  Tables<T> tb = cast_tables<T>(m->tab.t);
  FaceTopo ft = topo(m);
  T* trc = m->trc.as<T>();
  T* slot = m->slot.as<T>();
  T* hbuf = m->hbuf.as<T>();
  Fields<T> in;
  for (int k = 0; k < 5; ++k) {
    in.f[k] = q + k * m->N;
    in.scale[k] = 1;
  }
  DG_RUN(m, K_TRACE, st, k_trace<T, DIM, N, 5><<<trace_grid<DIM, N>(m->E), TraceShape<DIM, N>::THREADS, 0, st>>>(in, m->E, m->N, trc, m->S, tb));
  DG_RUN(m, K_FACE_EXPLICIT, st, k_face_explicit<T, DIM, N><<<grid_for(m->nF, 128), 128, 0, st>>>(ft, trc, slot, hbuf, tb, (T)ph.gamma,
                                                                                    (T)ph.lambda_min));
  if (m->nHC > 0)
    DG_RUN(m, K_HANG_GATHER, st, k_hang_gather<T, DIM, N, 9><<<grid_for(m->nHC * CS::NFP, 128), 128, 0, st>>>(ft, hbuf, slot, tb));
  DG_TILE(m, K_VOL_EXPLICIT,
          DG_RUN(m, K_VOL_EXPLICIT, st,
                 k_volume_explicit<T, DIM, N, M_><<<grid_for(m->E, CellShape<DIM, N, M_>::EPB),
                                                    CellShape<DIM, N, M_>::THREADS, 0, st>>>(
                     q, met_K<T>(m), met_invM<T>(m), slot, m->E, m->S, tb, ph, fns, fs,
                     m->terrain ? 1 : 0)));
  if (m->gll) {
    gl_convert<T, DIM, N>(m, fns, fns, 5, false, st);
    gl_convert<T, DIM, N>(m, fs, fs, 4, false, st);
  }
  DG_LAUNCH_CHECK("explicit operator");
  return DG_OK;
}

// per-Picard-iteration coefficients: h rho traces and the implicit Rusanov
// lambda coefficient at face points
template <typename T, int DIM, int N>
int Engine<T, DIM, N>::prepare(dg_mesh* m, const ImplK& ph, const T* rho, const T* plag, const T* ulag, int penalty,
                               cudaStream_t st) {
  int rc;
  if ((rc = far_ready(m)) != DG_OK) return rc;
  if ((rc = m->trc.ensure(sizeof(T) * 5 * m->S)) != DG_OK) return rc;
  if ((rc = m->slot.ensure(sizeof(T) * 9 * m->S)) != DG_OK) return rc;
  if ((rc = m->hbuf.ensure(sizeof(T) * 9 * (m->nH > 0 ? m->nH : 1))) != DG_OK) return rc;
  if ((rc = buf_trh<T>(m).ensure(sizeof(T) * m->S)) != DG_OK) return rc;
  if ((rc = buf_pcoef<T>(m).ensure(sizeof(T) * (m->nF > 0 ? m->nF : 1))) != DG_OK) return rc;
  if ((rc = m->wv.ensure(sizeof(T) * 6 * m->N)) != DG_OK) return rc;
  if ((rc = buf_irho<T>(m).ensure(sizeof(T) * m->N)) != DG_OK) return rc;
  if (m->gll) {   // GL copies of the frozen coefficients, used by every later call
    if ((rc = gl_buffers<T>(m)) != DG_OK) return rc;
    T* c = buf_gl<T>(m).template as<T>();
    gl_convert<T, DIM, N>(m, rho, c, 1, true, st);
    gl_convert<T, DIM, N>(m, plag, c + m->N, 1, true, st);
    gl_convert<T, DIM, N>(m, ulag, c + 2 * m->N, 3, true, st);
    rho = c;
    plag = c + m->N;
    ulag = c + 2 * m->N;
  }
  Tables<T> tb = cast_tables<T>(m->tab.t);
  FaceTopo ft = topo(m);
  DG_RUN(m, K_VEC, st, k_recip<T><<<grid_for(m->N, 256), 256, 0, st>>>(rho, buf_irho<T>(m).template as<T>(), m->N));
  Fields<T> in;
  in.f[0] = plag;
  in.scale[0] = (T)(ph.gamma / (ph.gamma - 1.0));
  DG_RUN(m, K_TRACE, st, k_trace<T, DIM, N, 1><<<trace_grid<DIM, N>(m->E), TraceShape<DIM, N>::THREADS, 0, st>>>(in, m->E, m->N, buf_trh<T>(m).template as<T>(), m->S, tb));
  if (penalty) {
    for (int c = 0; c < 3; ++c) {
      in.f[c] = ulag + c * m->N;
      in.scale[c] = 1;
    }
    DG_RUN(m, K_TRACE, st, k_trace<T, DIM, N, 3><<<trace_grid<DIM, N>(m->E), TraceShape<DIM, N>::THREADS, 0, st>>>(in, m->E, m->N, m->trc.as<T>(), m->S, tb));
    DG_RUN(m, K_FACE_LAMBDA, st, k_face_lambda<T, DIM, N><<<grid_for(m->nF, 128), 128, 0, st>>>(ft, m->trc.as<T>(), (T)(0.5 * ph.a_dt),
                                                                    buf_pcoef<T>(m).template as<T>(), tb));
    if ((rc = buf_pcs<T>(m).ensure(sizeof(T) * (m->S > 0 ? m->S : 1))) != DG_OK) return rc;
    DG_RUN(m, K_FACE_LAMBDA, st, k_pcoef_slots<T><<<grid_for(m->nF, 256), 256, 0, st>>>(
                                     m->fp_minus, m->fp_plus, m->nFar > 0 ? m->fp_far : nullptr,
                                     buf_pcoef<T>(m).template as<T>(), m->nF, buf_pcs<T>(m).template as<T>()));
  }
  DG_LAUNCH_CHECK("implicit coefficients");
  return DG_OK;
}

// y = S x (scaled Schur vmult); coefficients from prepare().  Two fused
// face + cell passes (gradient, divergence); 2:1 faces get their face
// values from the face kernels run on the hanging face points only.
template <typename T, int DIM, int N>
int Engine<T, DIM, N>::vmult(dg_mesh* m, const ImplK& ph, const T* rho, const T* plag, int penalty,
                             const T* x, T* y, cudaStream_t st) {
  using CS = CellShape<DIM, N>;
  using FS = FusedShape<DIM, N>;
  Tables<T> tb = cast_tables<T>(m->tab.t);
  const FaceTopo fh = topo_hanging(m);
  T* trc = m->trc.as<T>();
  T* slot = m->slot.as<T>();
  T* hbuf = m->hbuf.as<T>();
  T* wv = m->wv.as<T>();
  const T* snS = nullptr;
  int rc;
  if ((rc = fused_normals<T>(m, st, &snS)) != DG_OK) return rc;
  const bool hang = m->nHC > 0, stage = fused_stage<T>(m);
  const T* pcs = penalty ? buf_pcs<T>(m).template as<T>() : nullptr;
  if (m->gll) {   // coefficients from prepare's GL copies; x to the GL basis
    T* c = buf_gl<T>(m).template as<T>();
    plag = c + m->N;
    gl_convert<T, DIM, N>(m, x, c + 5 * m->N, 1, true, st);
    x = c + 5 * m->N;
  }
  Fields<T> in;
  in.f[0] = x;
  in.scale[0] = 1;
  if (hang || !stage)
    DG_RUN(m, K_TRACE, st, k_trace<T, DIM, N, 1><<<trace_grid<DIM, N>(m->E), TraceShape<DIM, N>::THREADS, 0, st>>>(in, m->E, m->N, trc, m->S, tb));
  if (hang) {
    DG_RUN(m, K_FACE_GRAD, st, k_face_grad<T, DIM, N><<<grid_for(m->nH, 128), 128, 0, st>>>(fh, trc, penalty ? buf_pcoef<T>(m).template as<T>() : nullptr,
                                                                  slot, hbuf, tb));
    DG_RUN(m, K_HANG_GATHER, st, k_hang_gather<T, DIM, N, DIM + 1><<<grid_for(m->nHC * CS::NFP, 128), 128, 0, st>>>(fh, hbuf, slot, tb));
  }
  const unsigned grid = grid_for(m->E, FS::EPB);
  // schedule 2: one thread per x-line (3D, degree 3, terrain-following
  // cells, 16-byte aligned vectors, 32-bit offsets); the gradient pass
  // leaves the face points' h rho w.n dS for the divergence pass in the
  // fifth field of the trace scratch (the traces of x and w use the first
  // three)
  const T* irho = buf_irho<T>(m).template as<T>();
  const bool lines = DIM == 3 && N == 4 && fused_sched<T>(m) == 2 && m->terrain &&
                     (!std::is_same<T, float>::value || m->tc32 != nullptr) && m->S <= (int64_t(1) << 29) &&
                     aligned16(x) && aligned16(y) && aligned16(wv) && aligned16(irho) && aligned16(plag);
  if constexpr (DIM == 3 && N == 4) {
    if (lines)
      DG_TILE(m, K_VOL_GRAD, {
        constexpr int EPB = line_epb<T>(M_);
        DG_RUN(m, K_VOL_GRAD, st, k_grad_lines<T, EPB><<<grid_for(m->E, EPB), LineShape<EPB>::THREADS, 0, st>>>(
                   x, m->cface, snS, pcs, irho, cell_geo<T>(m), slot, (int)m->E, (int)m->S, tb, ph, wv, y,
                   buf_trh<T>(m).template as<T>(), trc + 4 * m->S));
      })
  }
  if (lines)
    ;
  else if (stage)
    DG_RUN(m, K_VOL_GRAD, st, k_grad_fused<T, DIM, N, GRAD_VMULT, true><<<grid, FS::THREADS, 0, st>>>(
               x, trc, m->cface, snS, pcs, buf_irho<T>(m).template as<T>(), cell_geo<T>(m), slot, m->E, m->S, tb, ph,
               wv, y, nullptr, nullptr));
  else
    DG_RUN(m, K_VOL_GRAD, st, k_grad_fused<T, DIM, N, GRAD_VMULT, false><<<grid, FS::THREADS, 0, st>>>(
               x, trc, m->cface, snS, pcs, buf_irho<T>(m).template as<T>(), cell_geo<T>(m), slot, m->E, m->S, tb, ph,
               wv, y, nullptr, nullptr));
  Fields<T> w;
  for (int b = 0; b < DIM; ++b) {
    w.f[b] = wv + b * m->N;
    w.scale[b] = 1;
  }
  if (hang || !stage)
    DG_RUN(m, K_TRACE, st, k_trace<T, DIM, N, DIM><<<trace_grid<DIM, N>(m->E), TraceShape<DIM, N>::THREADS, 0, st>>>(w, m->E, m->N, trc, m->S, tb));
  if (hang) {
    DG_RUN(m, K_FACE_DIV, st, k_face_div<T, DIM, N><<<grid_for(m->nH, 128), 128, 0, st>>>(fh, trc, buf_trh<T>(m).template as<T>(), slot, hbuf, tb));
    DG_RUN(m, K_HANG_GATHER, st, k_hang_gather<T, DIM, N, 1><<<grid_for(m->nHC * CS::NFP, 128), 128, 0, st>>>(fh, hbuf, slot, tb));
  }
  if constexpr (DIM == 3 && N == 4) {
    if (lines)
      DG_TILE(m, K_VOL_DIV, {
        constexpr int EPB = line_epb<T>(M_);
        DG_RUN(m, K_VOL_DIV, st, k_div_lines<T, EPB><<<grid_for(m->E, EPB), LineShape<EPB>::THREADS, 0, st>>>(
                   w, trc + 4 * m->S, m->cface, plag, cell_geo<T>(m), slot, (int)m->E, tb, ph, y));
      })
  }
  if (lines)
    ;
  else if (stage)
    DG_RUN(m, K_VOL_DIV, st, k_div_fused<T, DIM, N, DIV_VMULT, true><<<grid, FS::THREADS, 0, st>>>(
               w, trc, buf_trh<T>(m).template as<T>(), m->cface, snS, plag, cell_geo<T>(m), slot, m->E, m->S, tb, ph,
               y, nullptr, nullptr, nullptr, nullptr));
  else
    DG_RUN(m, K_VOL_DIV, st, k_div_fused<T, DIM, N, DIV_VMULT, false><<<grid, FS::THREADS, 0, st>>>(
               w, trc, buf_trh<T>(m).template as<T>(), m->cface, snS, plag, cell_geo<T>(m), slot, m->E, m->S, tb, ph,
               y, nullptr, nullptr, nullptr, nullptr));
  if (m->gll) gl_convert<T, DIM, N>(m, y, y, 1, false, st);
  DG_LAUNCH_CHECK("schur vmult");
  return DG_OK;
}

// rhs of the scaled pressure system (uses wv[3N..6N) for u*)
template <typename T, int DIM, int N>
int Engine<T, DIM, N>::schur_rhs(dg_mesh* m, const ImplK& ph, const T* rho, const T* plag, const T* ulag,
                                 const T* mhat, const T* ehat, T* rhs, cudaStream_t st) {
  using CS = CellShape<DIM, N>;
  using FS = FusedShape<DIM, N>;
  Tables<T> tb = cast_tables<T>(m->tab.t);
  const FaceTopo fh = topo_hanging(m);
  T* trc = m->trc.as<T>();
  T* slot = m->slot.as<T>();
  T* hbuf = m->hbuf.as<T>();
  T* ustar = m->wv.as<T>() + 3 * m->N;
  const T* snS = nullptr;
  int rc;
  if ((rc = fused_normals<T>(m, st, &snS)) != DG_OK) return rc;
  const bool hang = m->nHC > 0, stage = fused_stage<T>(m);
  if (m->gll) {   // coefficients from prepare's GL copies; m_hat, e_hat to the GL basis
    T* c = buf_gl<T>(m).template as<T>();
    rho = c;
    plag = c + m->N;
    ulag = c + 2 * m->N;
    gl_convert<T, DIM, N>(m, mhat, c + 5 * m->N, 3, true, st);
    gl_convert<T, DIM, N>(m, ehat, c + 8 * m->N, 1, true, st);
    mhat = c + 5 * m->N;
    ehat = c + 8 * m->N;
  }
  if ((rc = far_predictors<T, DIM, N>(m, ph, mhat, ehat, st)) != DG_OK) return rc;
  ImplK pk = ph;
  pk.np = CS::NP;
  DG_RUN(m, K_USTAR, st, k_ustar<T><<<grid_for(m->N, 256), 256, 0, st>>>(mhat, rho, ulag, m->N, pk, ustar));
  Fields<T> w;
  for (int b = 0; b < DIM; ++b) {
    int c = DIM == 3 ? b : (b == 0 ? 0 : 2);
    w.f[b] = ustar + c * m->N;
    w.scale[b] = 1;
  }
  if (hang || !stage)
    DG_RUN(m, K_TRACE, st, k_trace<T, DIM, N, DIM><<<trace_grid<DIM, N>(m->E), TraceShape<DIM, N>::THREADS, 0, st>>>(w, m->E, m->N, trc, m->S, tb));
  if (hang) {
    DG_RUN(m, K_FACE_DIV, st, k_face_div<T, DIM, N><<<grid_for(m->nH, 128), 128, 0, st>>>(fh, trc, buf_trh<T>(m).template as<T>(), slot, hbuf, tb));
    DG_RUN(m, K_HANG_GATHER, st, k_hang_gather<T, DIM, N, 1><<<grid_for(m->nHC * CS::NFP, 128), 128, 0, st>>>(fh, hbuf, slot, tb));
  }
  const unsigned grid = grid_for(m->E, FS::EPB);
  if (stage)
    DG_RUN(m, K_VOL_DIV, st, k_div_fused<T, DIM, N, DIV_RHS, true><<<grid, FS::THREADS, 0, st>>>(
               w, trc, buf_trh<T>(m).template as<T>(), m->cface, snS, plag, cell_geo<T>(m), slot, m->E, m->S, tb, ph,
               rhs, ehat, rho, ulag, ustar));
  else
    DG_RUN(m, K_VOL_DIV, st, k_div_fused<T, DIM, N, DIV_RHS, false><<<grid, FS::THREADS, 0, st>>>(
               w, trc, buf_trh<T>(m).template as<T>(), m->cface, snS, plag, cell_geo<T>(m), slot, m->E, m->S, tb, ph,
               rhs, ehat, rho, ulag, ustar));
  if (m->gll) gl_convert<T, DIM, N>(m, rhs, rhs, 1, false, st);
  DG_LAUNCH_CHECK("schur rhs");
  return DG_OK;
}

// u = u* - a_dt w(p)
template <typename T, int DIM, int N>
int Engine<T, DIM, N>::recover(dg_mesh* m, const ImplK& ph, const T* rho, const T* ulag, const T* mhat,
                               const T* p, T* u, cudaStream_t st) {
  using CS = CellShape<DIM, N>;
  using FS = FusedShape<DIM, N>;
  Tables<T> tb = cast_tables<T>(m->tab.t);
  const FaceTopo fh = topo_hanging(m);
  T* trc = m->trc.as<T>();
  T* slot = m->slot.as<T>();
  T* hbuf = m->hbuf.as<T>();
  T* ustar = m->wv.as<T>() + 3 * m->N;
  const T* snS = nullptr;
  int rc;
  if ((rc = fused_normals<T>(m, st, &snS)) != DG_OK) return rc;
  const bool hang = m->nHC > 0, stage = fused_stage<T>(m);
  if (m->gll) {   // coefficients from prepare's GL copies; m_hat, p to the GL basis
    T* c = buf_gl<T>(m).template as<T>();
    rho = c;
    ulag = c + 2 * m->N;
    gl_convert<T, DIM, N>(m, mhat, c + 5 * m->N, 3, true, st);
    gl_convert<T, DIM, N>(m, p, c + 8 * m->N, 1, true, st);
    mhat = c + 5 * m->N;
    p = c + 8 * m->N;
  }
  {
    const T* no_ehat = nullptr;
    if ((rc = far_predictors<T, DIM, N>(m, ph, mhat, no_ehat, st)) != DG_OK) return rc;
  }
  ImplK pk = ph;
  pk.np = CS::NP;
  DG_RUN(m, K_USTAR, st, k_ustar<T><<<grid_for(m->N, 256), 256, 0, st>>>(mhat, rho, ulag, m->N, pk, ustar));
  Fields<T> in;
  in.f[0] = p;
  in.scale[0] = 1;
  if (hang || !stage)
    DG_RUN(m, K_TRACE, st, k_trace<T, DIM, N, 1><<<trace_grid<DIM, N>(m->E), TraceShape<DIM, N>::THREADS, 0, st>>>(in, m->E, m->N, trc, m->S, tb));
  if (hang) {
    DG_RUN(m, K_FACE_GRAD, st, k_face_grad<T, DIM, N><<<grid_for(m->nH, 128), 128, 0, st>>>(fh, trc, nullptr, slot, hbuf, tb));
    DG_RUN(m, K_HANG_GATHER, st, k_hang_gather<T, DIM, N, DIM + 1><<<grid_for(m->nHC * CS::NFP, 128), 128, 0, st>>>(fh, hbuf, slot, tb));
  }
  const unsigned grid = grid_for(m->E, FS::EPB);
  if (stage)
    DG_RUN(m, K_VOL_GRAD, st, k_grad_fused<T, DIM, N, GRAD_RECOVER, true><<<grid, FS::THREADS, 0, st>>>(
               p, trc, m->cface, snS, nullptr, buf_irho<T>(m).template as<T>(), cell_geo<T>(m), slot, m->E, m->S, tb,
               ph, nullptr, nullptr, ustar, u));
  else
    DG_RUN(m, K_VOL_GRAD, st, k_grad_fused<T, DIM, N, GRAD_RECOVER, false><<<grid, FS::THREADS, 0, st>>>(
               p, trc, m->cface, snS, nullptr, buf_irho<T>(m).template as<T>(), cell_geo<T>(m), slot, m->E, m->S, tb,
               ph, nullptr, nullptr, ustar, u));
  if (m->gll) gl_convert<T, DIM, N>(m, u, u, 3, false, st);
  DG_LAUNCH_CHECK("velocity recovery");
  return DG_OK;
}

int gl_basis(dg_mesh* m, const double* in, double* out, int nfld, bool to_gl, cudaStream_t st) {
  int rc;
  if ((rc = gl_buffers<double>(m)) != DG_OK) return rc;
  rc = DG_ERR_UNSUPPORTED;
  DG_DISPATCH(m, {
    gl_convert<double, D_, N_>(m, in, out, nfld, to_gl, st);
    rc = DG_OK;
  });
  if (rc == DG_OK) DG_LAUNCH_CHECK("nodal basis change");
  return rc;
}

double* gl_scratch(dg_mesh* m) {
  if (gl_buffers<double>(m) != DG_OK) return nullptr;
  return m->gl64.as<double>() + 5 * m->N;
}

template struct Engine<double, 2, 2>;
template struct Engine<double, 2, 3>;
template struct Engine<double, 2, 4>;
template struct Engine<double, 2, 5>;
template struct Engine<double, 3, 2>;
template struct Engine<double, 3, 3>;
template struct Engine<double, 3, 4>;
template struct Engine<double, 3, 5>;
template struct Engine<float, 2, 2>;
template struct Engine<float, 2, 3>;
template struct Engine<float, 2, 4>;
template struct Engine<float, 2, 5>;
template struct Engine<float, 3, 2>;
template struct Engine<float, 3, 3>;
template struct Engine<float, 3, 4>;
template struct Engine<float, 3, 5>;

// DG_PAIRS runs only the coefficient preparation and the vmult in pairs
#define DG_PAIRS_ENGINE(D, N)                                                                                   \
  template int Engine<df64, D, N>::prepare(dg_mesh*, const ImplK&, const df64*, const df64*, const df64*, int,  \
                                           cudaStream_t);                                                       \
  template int Engine<df64, D, N>::vmult(dg_mesh*, const ImplK&, const df64*, const df64*, int, const df64*,    \
                                         df64*, cudaStream_t);
DG_PAIRS_ENGINE(2, 2)
DG_PAIRS_ENGINE(2, 3)
DG_PAIRS_ENGINE(2, 4)
DG_PAIRS_ENGINE(2, 5)
DG_PAIRS_ENGINE(3, 2)
DG_PAIRS_ENGINE(3, 3)
DG_PAIRS_ENGINE(3, 4)
DG_PAIRS_ENGINE(3, 5)
#undef DG_PAIRS_ENGINE

__global__ void k_d2df(const double* __restrict__ a, df64* __restrict__ b, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) b[i] = df64(a[i]);
}

__global__ void k_df2d(const df64* __restrict__ a, double* __restrict__ b, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) b[i] = (double)a[i];
}

int to_pairs(dg_mesh* m, const double* a, df64* b, int64_t n, cudaStream_t st) {
  if (n > 0) DG_RUN(m, K_VEC, st, k_d2df<<<grid_for(n, 256), 256, 0, st>>>(a, b, n));
  DG_LAUNCH_CHECK("pair conversion");
  return DG_OK;
}

int from_pairs(dg_mesh* m, const df64* a, double* b, int64_t n, cudaStream_t st) {
  if (n > 0) DG_RUN(m, K_VEC, st, k_df2d<<<grid_for(n, 256), 256, 0, st>>>(a, b, n));
  DG_LAUNCH_CHECK("pair conversion");
  return DG_OK;
}

int ensure_pairs_geometry(dg_mesh* m, cudaStream_t st) {
  if (m->snSdf.p) return DG_OK;
  const double* snS = nullptr;
  int rc;
  if ((rc = fused_normals<double>(m, st, &snS)) != DG_OK) return rc;
  const int64_t nK = (int64_t)m->dim * m->dim * m->N, nG = (int64_t)(m->dim + 1) * m->nF, nS = m->dim * m->S;
  if ((rc = m->Kdf.ensure(sizeof(df64) * nK)) != DG_OK) return rc;
  if ((rc = m->invMdf.ensure(sizeof(df64) * m->N)) != DG_OK) return rc;
  if ((rc = m->fgeodf.ensure(sizeof(df64) * (nG > 0 ? nG : 1))) != DG_OK) return rc;
  if ((rc = to_pairs(m, m->K, m->Kdf.as<df64>(), nK, st)) != DG_OK) return rc;
  if ((rc = to_pairs(m, m->invM, m->invMdf.as<df64>(), m->N, st)) != DG_OK) return rc;
  if ((rc = to_pairs(m, m->fgeo, m->fgeodf.as<df64>(), nG, st)) != DG_OK) return rc;
  // the per-slot normals last: their buffer marks the geometry as made
  if ((rc = m->snSdf.ensure(sizeof(df64) * (nS > 0 ? nS : 1))) != DG_OK) return rc;
  return to_pairs(m, snS, m->snSdf.as<df64>(), nS, st);
}

}  // namespace dg

using namespace dg;

static int check_common(dg_ctx* ctx, const dg_mesh* m, const dg_phys* ph, const char* who) {
  if (!ctx || !m || !ph) {
    set_error("%s: NULL argument", who);
    return DG_ERR_ARG;
  }
  if (!(ph->gamma > 1.0)) {
    set_error("%s: gamma must be > 1", who);
    return DG_ERR_ARG;
  }
  if (!(ph->lambda_min >= 0.0)) {
    set_error("%s: lambda_min must be >= 0", who);
    return DG_ERR_ARG;
  }
  if (ph->precision != DG_FP64 && ph->precision != DG_MIXED && ph->precision != DG_MIXED_EXPLICIT &&
      ph->precision != DG_PAIRS) {
    set_error("%s: precision must be DG_FP64, DG_MIXED, DG_MIXED_EXPLICIT or DG_PAIRS", who);
    return DG_ERR_ARG;
  }
  if (ph->variant != DG_R1 && ph->variant != DG_R2) {
    set_error("%s: variant must be DG_R1 or DG_R2", who);
    return DG_ERR_ARG;
  }
  return DG_OK;
}

ImplK dg::impl_consts(const dg_phys* ph, double a_dt) {
  ImplK k;
  k.gamma = ph->gamma;
  k.g = ph->g;
  k.f = ph->f;
  k.a_dt = a_dt;
  k.r2 = ph->variant == DG_R2;
  k.fcell = ph->f_cell;
  k.np = 1;
  k.gamma_f = (float)ph->gamma;
  k.g_f = (float)ph->g;
  k.adt_f = (float)a_dt;
  k.f_f = (float)ph->f;
  k.fcell32 = nullptr;
  k.penalty = ph->penalty ? 1 : 0;
  const double beta = a_dt * ph->f;
  k.dbeta = 1.0 / (1.0 + beta * beta);
  k.cgrav = (ph->gamma - 1.0) * a_dt * a_dt * ph->g;
  k.dbeta_f = (float)k.dbeta;
  k.cgrav_f = (float)k.cgrav;
  k.gamma_p = df64(ph->gamma);
  k.g_p = df64(ph->g);
  k.adt_p = df64(a_dt);
  k.beta_p = df64(beta);
  k.dbeta_p = df64(k.dbeta);
  k.cgrav_p = df64(k.cgrav);
  return k;
}

extern "C" {

int dg_mesh_set_far_state(dg_ctx* ctx, dg_mesh* mesh, const double* q_far, void* stream) {
  if (!ctx || !mesh || !q_far) {
    set_error("dg_mesh_set_far_state: NULL argument");
    return DG_ERR_ARG;
  }
  if (mesh->nFar == 0) return DG_OK;
  int rc = DG_ERR_UNSUPPORTED;
  DG_DISPATCH(mesh, rc = (set_far_state<D_, N_>(mesh, q_far, (cudaStream_t)stream)));
  return rc;
}

int dg_apply_explicit(dg_ctx* ctx, const dg_mesh* mesh, const dg_phys* ph, const double* q, double* fns,
                      double* fs, void* stream) {
  int rc = check_common(ctx, mesh, ph, "dg_apply_explicit");
  if (rc) return rc;
  if (!q || !fns || !fs) {
    set_error("dg_apply_explicit: NULL array");
    return DG_ERR_ARG;
  }
  PhysK k{ph->gamma, ph->g, ph->f, ph->f_cell, ph->lambda_min};
  dg_mesh* m = const_cast<dg_mesh*>(mesh);
  if (ph->precision == DG_MIXED_EXPLICIT) {
    if (m->nFar > 0 || m->gll) {
      set_error("dg_apply_explicit: DG_MIXED_EXPLICIT is not implemented with far-field faces or Gauss-Lobatto nodes");
      return DG_ERR_UNSUPPORTED;
    }
    if (!m->bg_set) {
      set_error("dg_apply_explicit: DG_MIXED_EXPLICIT needs a background (dg_mesh_set_background)");
      return DG_ERR_ARG;
    }
    rc = explicit_mixed(m, k, q, fns, fs, (cudaStream_t)stream);
  } else {
    rc = DG_ERR_UNSUPPORTED;
    DG_DISPATCH(m, rc = (Engine<double, D_, N_>::explicit_rates(m, k, q, fns, fs, (cudaStream_t)stream)));
  }
  if (rc != DG_OK) return rc;
  return sponge_rt(m, q, fns, (cudaStream_t)stream);
}

int dg_apply_implicit(dg_ctx* ctx, const dg_mesh* mesh, const dg_phys* ph, const dg_implicit_coeffs* cf,
                      const double* x, double* y, void* stream) {
  int rc = check_common(ctx, mesh, ph, "dg_apply_implicit");
  if (rc) return rc;
  if (!cf || !cf->rho || !cf->p_lag || !cf->u_lag || !x || !y || x == y) {
    set_error("dg_apply_implicit: NULL or aliased array");
    return DG_ERR_ARG;
  }
  dg_mesh* m = const_cast<dg_mesh*>(mesh);
  ImplK k = impl_consts(ph, cf->a_dt);
  cudaStream_t st = (cudaStream_t)stream;
  if (ph->precision == DG_PAIRS)
    return schur_vmult_pairs(m, k, cf->rho, cf->p_lag, cf->u_lag, ph->penalty, x, y, st);
  if (ph->precision != DG_FP64)
    return schur_vmult_mixed(m, k, cf->rho, cf->p_lag, cf->u_lag, ph->penalty, x, y, st);
  DG_DISPATCH(m, {
    using EN = Engine<double, D_, N_>;
    if ((rc = EN::prepare(m, k, cf->rho, cf->p_lag, cf->u_lag, ph->penalty, st)) != DG_OK) return rc;
    return EN::vmult(m, k, cf->rho, cf->p_lag, ph->penalty, x, y, st);
  });
  return DG_ERR_UNSUPPORTED;
}

int dg_schur_rhs(dg_ctx* ctx, const dg_mesh* mesh, const dg_phys* ph, const dg_implicit_coeffs* cf,
                 const double* mhat, const double* ehat, double* rhs, void* stream) {
  int rc = check_common(ctx, mesh, ph, "dg_schur_rhs");
  if (rc) return rc;
  if (!cf || !cf->rho || !cf->p_lag || !cf->u_lag || !mhat || !ehat || !rhs) {
    set_error("dg_schur_rhs: NULL array");
    return DG_ERR_ARG;
  }
  dg_mesh* m = const_cast<dg_mesh*>(mesh);
  ImplK k = impl_consts(ph, cf->a_dt);
  cudaStream_t st = (cudaStream_t)stream;
  DG_DISPATCH(m, {
    using EN = Engine<double, D_, N_>;
    // the penalty's lambda enters the far-field outer data
    const int pen = m->nFar > 0 ? ph->penalty : 0;
    if ((rc = EN::prepare(m, k, cf->rho, cf->p_lag, cf->u_lag, pen, st)) != DG_OK) return rc;
    return EN::schur_rhs(m, k, cf->rho, cf->p_lag, cf->u_lag, mhat, ehat, rhs, st);
  });
  return DG_ERR_UNSUPPORTED;
}

int dg_recover_velocity(dg_ctx* ctx, const dg_mesh* mesh, const dg_phys* ph, const dg_implicit_coeffs* cf,
                        const double* mhat, const double* p, double* u, void* stream) {
  int rc = check_common(ctx, mesh, ph, "dg_recover_velocity");
  if (rc) return rc;
  if (!cf || !cf->rho || !cf->u_lag || !mhat || !p || !u) {
    set_error("dg_recover_velocity: NULL array");
    return DG_ERR_ARG;
  }
  dg_mesh* m = const_cast<dg_mesh*>(mesh);
  ImplK k = impl_consts(ph, cf->a_dt);
  cudaStream_t st = (cudaStream_t)stream;
  DG_DISPATCH(m, {
    using EN = Engine<double, D_, N_>;
    if ((rc = EN::prepare(m, k, cf->rho, cf->p_lag ? cf->p_lag : p, cf->u_lag, 0, st)) != DG_OK) return rc;
    return EN::recover(m, k, cf->rho, cf->u_lag, mhat, p, u, st);
  });
  return DG_ERR_UNSUPPORTED;
}

}  // extern "C"
