// Launch sequences of the explicit operator, the Schur-complement vmult,
// the Schur right-hand side and the velocity recovery, plus their C entry
// points.
#include "engine.cuh"

namespace dg {

template <typename T, int DIM, int N>
int Engine<T, DIM, N>::explicit_rates(dg_mesh* m, const PhysK& ph, const T* q, T* fns, T* fs,
                                      cudaStream_t st) {
  using CS = CellShape<DIM, N>;
  int rc;
  if ((rc = m->trc.ensure(sizeof(T) * 5 * m->S)) != DG_OK) return rc;
  if ((rc = m->slot.ensure(sizeof(T) * 9 * m->S)) != DG_OK) return rc;
  if ((rc = m->hbuf.ensure(sizeof(T) * 9 * (m->nH > 0 ? m->nH : 1))) != DG_OK) return rc;
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
  DG_LAUNCH_CHECK("explicit operator");
  return DG_OK;
}

// per-Picard-iteration coefficients: h rho traces and the implicit Rusanov
// lambda coefficient at face points
template <typename T, int DIM, int N>
int Engine<T, DIM, N>::prepare(dg_mesh* m, const ImplK& ph, const T* rho, const T* plag, const T* ulag, int penalty,
                               cudaStream_t st) {
  int rc;
  if ((rc = m->trc.ensure(sizeof(T) * 5 * m->S)) != DG_OK) return rc;
  if ((rc = m->slot.ensure(sizeof(T) * 9 * m->S)) != DG_OK) return rc;
  if ((rc = m->hbuf.ensure(sizeof(T) * 9 * (m->nH > 0 ? m->nH : 1))) != DG_OK) return rc;
  if ((rc = buf_trh<T>(m).ensure(sizeof(T) * m->S)) != DG_OK) return rc;
  if ((rc = buf_pcoef<T>(m).ensure(sizeof(T) * (m->nF > 0 ? m->nF : 1))) != DG_OK) return rc;
  if ((rc = m->wv.ensure(sizeof(T) * 6 * m->N)) != DG_OK) return rc;
  if ((rc = buf_irho<T>(m).ensure(sizeof(T) * m->N)) != DG_OK) return rc;
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
  }
  DG_LAUNCH_CHECK("implicit coefficients");
  return DG_OK;
}

// y = S x (scaled Schur vmult); coefficients from prepare()
template <typename T, int DIM, int N>
int Engine<T, DIM, N>::vmult(dg_mesh* m, const ImplK& ph, const T* rho, const T* plag, int penalty,
                             const T* x, T* y, cudaStream_t st) {
  using CS = CellShape<DIM, N>;
  Tables<T> tb = cast_tables<T>(m->tab.t);
  FaceTopo ft = topo(m);
  T* trc = m->trc.as<T>();
  T* slot = m->slot.as<T>();
  T* hbuf = m->hbuf.as<T>();
  T* wv = m->wv.as<T>();
  Fields<T> in;
  in.f[0] = x;
  in.scale[0] = 1;
  DG_RUN(m, K_TRACE, st, k_trace<T, DIM, N, 1><<<trace_grid<DIM, N>(m->E), TraceShape<DIM, N>::THREADS, 0, st>>>(in, m->E, m->N, trc, m->S, tb));
  DG_RUN(m, K_FACE_GRAD, st, k_face_grad<T, DIM, N><<<grid_for(m->nF, 128), 128, 0, st>>>(ft, trc, penalty ? buf_pcoef<T>(m).template as<T>() : nullptr,
                                                                slot, hbuf, tb));
  if (m->nHC > 0)
    DG_RUN(m, K_HANG_GATHER, st, k_hang_gather<T, DIM, N, DIM + 1><<<grid_for(m->nHC * CS::NFP, 128), 128, 0, st>>>(ft, hbuf, slot, tb));
  DG_TILE(m, K_VOL_GRAD,
          DG_RUN(m, K_VOL_GRAD, st,
                 k_volume_grad<T, DIM, N, GRAD_VMULT, M_><<<grid_for(m->E, CellShape<DIM, N, M_>::EPB),
                                                          CellShape<DIM, N, M_>::THREADS, 0, st>>>(
                     x, buf_irho<T>(m).template as<T>(), cell_geo<T>(m), slot, m->E, m->S, tb, ph, wv, y, nullptr, nullptr)));
  Fields<T> w;
  for (int b = 0; b < DIM; ++b) {
    w.f[b] = wv + b * m->N;
    w.scale[b] = 1;
  }
  DG_RUN(m, K_TRACE, st, k_trace<T, DIM, N, DIM><<<trace_grid<DIM, N>(m->E), TraceShape<DIM, N>::THREADS, 0, st>>>(w, m->E, m->N, trc, m->S, tb));
  DG_RUN(m, K_FACE_DIV, st, k_face_div<T, DIM, N><<<grid_for(m->nF, 128), 128, 0, st>>>(ft, trc, buf_trh<T>(m).template as<T>(), slot, hbuf, tb));
  if (m->nHC > 0)
    DG_RUN(m, K_HANG_GATHER, st, k_hang_gather<T, DIM, N, 1><<<grid_for(m->nHC * CS::NFP, 128), 128, 0, st>>>(ft, hbuf, slot, tb));
  DG_TILE(m, K_VOL_DIV,
          DG_RUN(m, K_VOL_DIV, st,
                 k_volume_div<T, DIM, N, DIV_VMULT, M_><<<grid_for(m->E, CellShape<DIM, N, M_>::EPB),
                                                         CellShape<DIM, N, M_>::THREADS, 0, st>>>(
                     w, plag, cell_geo<T>(m), slot, m->E, m->S, tb, ph, y, nullptr, nullptr, nullptr,
                     nullptr)));
  DG_LAUNCH_CHECK("schur vmult");
  return DG_OK;
}

// rhs of the scaled pressure system (uses wv[3N..6N) for u*)
template <typename T, int DIM, int N>
int Engine<T, DIM, N>::schur_rhs(dg_mesh* m, const ImplK& ph, const T* rho, const T* plag, const T* ulag,
                                 const T* mhat, const T* ehat, T* rhs, cudaStream_t st) {
  using CS = CellShape<DIM, N>;
  Tables<T> tb = cast_tables<T>(m->tab.t);
  FaceTopo ft = topo(m);
  T* trc = m->trc.as<T>();
  T* slot = m->slot.as<T>();
  T* hbuf = m->hbuf.as<T>();
  T* ustar = m->wv.as<T>() + 3 * m->N;
  ImplK pk = ph;
  pk.np = CS::NP;
  DG_RUN(m, K_USTAR, st, k_ustar<T><<<grid_for(m->N, 256), 256, 0, st>>>(mhat, rho, ulag, m->N, pk, ustar));
  Fields<T> w;
  for (int b = 0; b < DIM; ++b) {
    int c = DIM == 3 ? b : (b == 0 ? 0 : 2);
    w.f[b] = ustar + c * m->N;
    w.scale[b] = 1;
  }
  DG_RUN(m, K_TRACE, st, k_trace<T, DIM, N, DIM><<<trace_grid<DIM, N>(m->E), TraceShape<DIM, N>::THREADS, 0, st>>>(w, m->E, m->N, trc, m->S, tb));
  DG_RUN(m, K_FACE_DIV, st, k_face_div<T, DIM, N><<<grid_for(m->nF, 128), 128, 0, st>>>(ft, trc, buf_trh<T>(m).template as<T>(), slot, hbuf, tb));
  if (m->nHC > 0)
    DG_RUN(m, K_HANG_GATHER, st, k_hang_gather<T, DIM, N, 1><<<grid_for(m->nHC * CS::NFP, 128), 128, 0, st>>>(ft, hbuf, slot, tb));
  DG_TILE(m, K_VOL_DIV,
          DG_RUN(m, K_VOL_DIV, st,
                 k_volume_div<T, DIM, N, DIV_RHS, M_><<<grid_for(m->E, CellShape<DIM, N, M_>::EPB),
                                                       CellShape<DIM, N, M_>::THREADS, 0, st>>>(
                     w, plag, cell_geo<T>(m), slot, m->E, m->S, tb, ph, rhs, ehat, rho, ulag, ustar)));
  DG_LAUNCH_CHECK("schur rhs");
  return DG_OK;
}

// u = u* - a_dt w(p)
template <typename T, int DIM, int N>
int Engine<T, DIM, N>::recover(dg_mesh* m, const ImplK& ph, const T* rho, const T* ulag, const T* mhat,
                               const T* p, T* u, cudaStream_t st) {
  using CS = CellShape<DIM, N>;
  Tables<T> tb = cast_tables<T>(m->tab.t);
  FaceTopo ft = topo(m);
  T* trc = m->trc.as<T>();
  T* slot = m->slot.as<T>();
  T* hbuf = m->hbuf.as<T>();
  T* ustar = m->wv.as<T>() + 3 * m->N;
  ImplK pk = ph;
  pk.np = CS::NP;
  DG_RUN(m, K_USTAR, st, k_ustar<T><<<grid_for(m->N, 256), 256, 0, st>>>(mhat, rho, ulag, m->N, pk, ustar));
  Fields<T> in;
  in.f[0] = p;
  in.scale[0] = 1;
  DG_RUN(m, K_TRACE, st, k_trace<T, DIM, N, 1><<<trace_grid<DIM, N>(m->E), TraceShape<DIM, N>::THREADS, 0, st>>>(in, m->E, m->N, trc, m->S, tb));
  DG_RUN(m, K_FACE_GRAD, st, k_face_grad<T, DIM, N><<<grid_for(m->nF, 128), 128, 0, st>>>(ft, trc, nullptr, slot, hbuf, tb));
  if (m->nHC > 0)
    DG_RUN(m, K_HANG_GATHER, st, k_hang_gather<T, DIM, N, DIM + 1><<<grid_for(m->nHC * CS::NFP, 128), 128, 0, st>>>(ft, hbuf, slot, tb));
  DG_TILE(m, K_VOL_GRAD,
          DG_RUN(m, K_VOL_GRAD, st,
                 k_volume_grad<T, DIM, N, GRAD_RECOVER, M_><<<grid_for(m->E, CellShape<DIM, N, M_>::EPB),
                                                            CellShape<DIM, N, M_>::THREADS, 0, st>>>(
                     p, buf_irho<T>(m).template as<T>(), cell_geo<T>(m), slot, m->E, m->S, tb, ph, nullptr, nullptr, ustar, u)));
  DG_LAUNCH_CHECK("velocity recovery");
  return DG_OK;
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
  if (ph->precision != DG_FP64 && ph->precision != DG_MIXED && ph->precision != DG_MIXED_EXPLICIT) {
    set_error("%s: precision must be DG_FP64, DG_MIXED or DG_MIXED_EXPLICIT", who);
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
  const double beta = a_dt * ph->f;
  k.dbeta = 1.0 / (1.0 + beta * beta);
  k.cgrav = (ph->gamma - 1.0) * a_dt * a_dt * ph->g;
  k.dbeta_f = (float)k.dbeta;
  k.cgrav_f = (float)k.cgrav;
  return k;
}

extern "C" {

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
    if ((rc = EN::prepare(m, k, cf->rho, cf->p_lag, cf->u_lag, 0, st)) != DG_OK) return rc;
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
