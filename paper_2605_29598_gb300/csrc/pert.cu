// Perturbation form of the explicit operator for the mixed-precision path.
//
// With a background state qb (FP64, set once per mesh), the rates are
//   F(q) = F(qb) + [F(q) - F(qb)].
// F(qb) is computed once in FP64.  The difference is evaluated in FP32 from
// the perturbation q' = q - qb (the subtraction in FP64, then rounded) by
// expanding every nonlinear flux so that no large background term cancels:
//   u' = (m' - ub rho') / rho,          (rho kappa)' = (mb.u' + m'.ub + m'.u') / 2,
//   p' = (gamma - 1)(E' - (rho kappa)'),  (a u)' = ab u' + a' ub + a' u'.
// The Rusanov term lambda/2 [a] - lambdab/2 [ab] becomes
//   lambda/2 [a'] + (lambda - lambdab)/2 [ab],
// with the background jumps [ab] and lambdab taken from FP64 once.
#include <cmath>

#include "engine.cuh"

namespace dg {

// background jumps at face points (FP64 -> FP32): rho, m_x, m_y, m_z,
// rho kappa, p (minus side minus plus side), and lambdab |n dS| / 2
template <int DIM, int N>
__global__ void k_bg_jumps(FaceTopo ft, const double* __restrict__ trc, Tables<double> tb, double gamma,
                           float* __restrict__ jump) {
  int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= ft.nF) return;
  const int64_t S = ft.S, nF = ft.nF;
  int sm = ft.fp_minus[p], code = ft.fp_plus[p];
  double qm[5], qp[5], nS[DIM], n2 = 0;
  for (int b = 0; b < DIM; ++b) {
    nS[b] = ft.fgeo[b * nF + p];
    n2 += nS[b] * nS[b];
  }
  for (int q = 0; q < 5; ++q) qm[q] = trc[q * S + sm];
  if (code == -1) {
    double mn = 0;
    for (int b = 0; b < DIM; ++b) mn += qm[1 + comp_of<DIM>(b)] * nS[b];
    mn /= n2;
    for (int q = 0; q < 5; ++q) qp[q] = qm[q];
    for (int b = 0; b < DIM; ++b) qp[1 + comp_of<DIM>(b)] -= 2 * mn * nS[b];
  } else {
    for (int q = 0; q < 5; ++q) qp[q] = plus_value<double, DIM, N>(ft, tb, trc + q * S, code, qm[q]);
  }
  double rkm = 0.5 * (qm[1] * qm[1] + qm[2] * qm[2] + qm[3] * qm[3]) / qm[0];
  double rkp = 0.5 * (qp[1] * qp[1] + qp[2] * qp[2] + qp[3] * qp[3]) / qp[0];
  double pm = (gamma - 1) * (qm[4] - rkm), pp = (gamma - 1) * (qp[4] - rkp);
  double unm = 0, unp = 0;
  for (int b = 0; b < DIM; ++b) {
    unm += qm[1 + comp_of<DIM>(b)] / qm[0] * nS[b];
    unp += qp[1 + comp_of<DIM>(b)] / qp[0] * nS[b];
  }
  const double j[7] = {qm[0] - qp[0], qm[1] - qp[1], qm[2] - qp[2], qm[3] - qp[3], rkm - rkp, pm - pp,
                       0.5 * fmax(fabs(unm), fabs(unp))};
  for (int k = 0; k < 7; ++k) jump[k * nF + p] = (float)j[k];
}

// q' = q - qb in FP64, rounded to FP32
__global__ void k_perturbation(const double* __restrict__ q, const double* __restrict__ qb, int64_t n5,
                               float* __restrict__ qp) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n5) qp[i] = (float)(q[i] - qb[i]);
}

// F = F(qb) + F' (FP64 result)
__global__ void k_add_rates(const double* __restrict__ fb, const float* __restrict__ fp, int64_t n,
                            double* __restrict__ out) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) out[i] = fb[i] + (double)fp[i];
}

__global__ void k_bg_cast(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}

// pointwise perturbation primitives
struct PertPrim {
  float ub[3], up[3];        // background velocity, velocity perturbation
  float rkb, rkp;            // (rho kappa) background, perturbation
  float pb, pp;              // pressure background, perturbation
};

__device__ __forceinline__ PertPrim pert_prim(const float qb[5], const float qp[5], float gm1) {
  PertPrim o;
  const float irb = 1.f / qb[0], ir = 1.f / (qb[0] + qp[0]);
  for (int c = 0; c < 3; ++c) {
    o.ub[c] = qb[1 + c] * irb;
    o.up[c] = (qp[1 + c] - o.ub[c] * qp[0]) * ir;
  }
  o.rkb = 0.5f * (qb[1] * o.ub[0] + qb[2] * o.ub[1] + qb[3] * o.ub[2]);
  o.rkp = 0.5f * (qb[1] * o.up[0] + qb[2] * o.up[1] + qb[3] * o.up[2] + qp[1] * o.ub[0] + qp[2] * o.ub[1] +
                  qp[3] * o.ub[2] + qp[1] * o.up[0] + qp[2] * o.up[1] + qp[3] * o.up[2]);
  o.pb = gm1 * (qb[4] - o.rkb);
  o.pp = gm1 * (qp[4] - o.rkp);
  return o;
}

// perturbation numerical fluxes at face points (slot fields as in the FP64
// operator: 0..4 non-stiff, 5..8 stiff)
template <int DIM, int N>
__global__ void k_face_explicit_pert(FaceTopo ft, const float* __restrict__ trp, const float* __restrict__ trb,
                                     const float* __restrict__ jump, float* __restrict__ slot,
                                     float* __restrict__ hbuf, Tables<float> tb, float gamma,
                                     float lambda_min) {
  int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= ft.nF) return;
  const int64_t S = ft.S, nF = ft.nF, nH = ft.nH;
  const int sm = __ldg(ft.fp_minus + p), code = __ldg(ft.fp_plus + p);
  float nS[DIM], n2 = 0;
#pragma unroll
  for (int b = 0; b < DIM; ++b) {
    nS[b] = __ldg(ft.fgeo32 + b * nF + p);
    n2 += nS[b] * nS[b];
  }
  float bm[5], bp[5], pm_[5], pp_[5];
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    bm[q] = __ldg(trb + q * S + sm);
    pm_[q] = __ldg(trp + q * S + sm);
  }
  if (code == -1) {
    // mirror state of the full state: m+ = m- - 2 (m-.n) n, linear, so it
    // applies to background and perturbation separately
    float mb = 0, mp = 0;
#pragma unroll
    for (int b = 0; b < DIM; ++b) {
      mb += bm[1 + comp_of<DIM>(b)] * nS[b];
      mp += pm_[1 + comp_of<DIM>(b)] * nS[b];
    }
    mb /= n2;
    mp /= n2;
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      bp[q] = bm[q];
      pp_[q] = pm_[q];
    }
#pragma unroll
    for (int b = 0; b < DIM; ++b) {
      bp[1 + comp_of<DIM>(b)] -= 2 * mb * nS[b];
      pp_[1 + comp_of<DIM>(b)] -= 2 * mp * nS[b];
    }
  } else {
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      bp[q] = plus_value<float, DIM, N>(ft, tb, trb + q * S, code, bm[q]);
      pp_[q] = plus_value<float, DIM, N>(ft, tb, trp + q * S, code, pm_[q]);
    }
  }
  const float gm1 = gamma - 1.f;
  const PertPrim A = pert_prim(bm, pm_, gm1), B = pert_prim(bp, pp_, gm1);
  float unbA = 0, unpA = 0, unbB = 0, unpB = 0;
#pragma unroll
  for (int b = 0; b < DIM; ++b) {
    const int c = comp_of<DIM>(b);
    unbA += A.ub[c] * nS[b];
    unpA += A.up[c] * nS[b];
    unbB += B.ub[c] * nS[b];
    unpB += B.up[c] * nS[b];
  }
  // lambda |n dS| / 2 of the full state and of the background
  const float pen = 0.5f * fmaxf(fabsf(unbA + unpA), fabsf(unbB + unpB));
  // background jumps and lambda from FP64 (walls included: mirror state)
  float jb[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) jb[k] = __ldg(jump + k * nF + p);
  const float pbar = __ldg(jump + 6 * nF + p);
  const float dpen = pen - pbar;
  // non-stiff terms: both coefficients floored at lambda_min |n dS| / 2
  const float pfl = 0.5f * lambda_min * sqrtf(n2);
  const float pns = lambda_min > 0.f ? fmaxf(pen, pfl) : pen;
  const float dpns = lambda_min > 0.f ? pns - fmaxf(pbar, pfl) : dpen;
  // products (a u.n)' = ab un' + a' unb + a' un'
  auto prod = [](float ab, float ap, float unb, float unp) { return ab * unp + ap * unb + ap * unp; };
  float mnA = 0.f, mnB = 0.f;   // m'.n dS on both sides (the mass flux is linear)
#pragma unroll
  for (int b = 0; b < DIM; ++b) {
    mnA += pm_[1 + comp_of<DIM>(b)] * nS[b];
    mnB += pp_[1 + comp_of<DIM>(b)] * nS[b];
  }
  put<float>(slot, hbuf, S, nH, 0, sm, code, 0.5f * (mnA + mnB) + pns * (pm_[0] - pp_[0]) + dpns * jb[0]);
#pragma unroll
  for (int c = 0; c < 3; ++c)
    put<float>(slot, hbuf, S, nH, 1 + c, sm, code,
               0.5f * (prod(bm[1 + c], pm_[1 + c], unbA, unpA) + prod(bp[1 + c], pp_[1 + c], unbB, unpB)) +
                   pns * (pm_[1 + c] - pp_[1 + c]) + dpns * jb[1 + c]);
  put<float>(slot, hbuf, S, nH, 4, sm, code,
             0.5f * (prod(A.rkb, A.rkp, unbA, unpA) + prod(B.rkb, B.rkp, unbB, unpB)) +
                 pns * (A.rkp - B.rkp) + dpns * jb[4]);
  const float pav = 0.5f * (A.pp + B.pp);
  put<float>(slot, hbuf, S, nH, 5, sm, code, pav * nS[0]);
  put<float>(slot, hbuf, S, nH, 6, sm, code, DIM == 3 ? pav * nS[DIM == 3 ? 1 : 0] : 0.f);
  put<float>(slot, hbuf, S, nH, 7, sm, code, pav * nS[DIM - 1]);
  put<float>(slot, hbuf, S, nH, 8, sm, code,
             0.5f * gamma / gm1 * (prod(A.pb, A.pp, unbA, unpA) + prod(B.pb, B.pp, unbB, unpB)) +
                 (pen * (A.pp - B.pp) + dpen * jb[5]) / gm1);
}

// perturbation cell integrals + lift + inverse mass, FP32 rates F'
template <int DIM, int N>
__global__ void __launch_bounds__(CellShape<DIM, N>::THREADS)
k_volume_explicit_pert(const float* __restrict__ qp, const float* __restrict__ qb, CellGeo<float> geo,
                       const float* __restrict__ slot, int64_t E, int64_t S, Tables<float> tb, float gamma,
                       float g, float f, const float* __restrict__ fcell32, float* __restrict__ fns,
                       float* __restrict__ fs) {
  using CS = CellShape<DIM, N>;
  constexpr int NP = CS::NP, EPB = CS::EPB;
  __shared__ float sm[EPB][DIM][NP];
  const int le = threadIdx.x / NP, i = threadIdx.x % NP;
  const int64_t e = (int64_t)blockIdx.x * EPB + le;
  const bool active = e < E;
  const int64_t Nn = E * NP;
  const int64_t node = active ? e * NP + i : 0;
  int idx[3];
  node_index<DIM, N>(i, idx);
  float b5[5] = {1.f, 0.f, 0.f, 0.f, 1.f}, p5[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
  float K[DIM][DIM], iM = 0.f;
  __shared__ float sxw[2 * N];
  stage_nodes<float, N>(geo, sxw);
  __syncthreads();
  if (active) {
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      b5[q] = __ldg(qb + q * Nn + node);
      p5[q] = __ldg(qp + q * Nn + node);
    }
    node_metric<float, DIM, N>(geo, e, node, Nn, idx, K, iM, sxw);
  } else {
#pragma unroll
    for (int a = 0; a < DIM; ++a)
#pragma unroll
      for (int b = 0; b < DIM; ++b) K[a][b] = 0.f;
  }
  const float gm1 = gamma - 1.f;
  const PertPrim P = pert_prim(b5, p5, gm1);
  const float hb = gamma / gm1 * P.pb, hp = gamma / gm1 * P.pp;
  float utb[DIM], utp[DIM], mtp[DIM];   // contravariant (times w det J) ub, u', m'
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    utb[a] = 0.f;
    utp[a] = 0.f;
    mtp[a] = 0.f;
#pragma unroll
    for (int b = 0; b < DIM; ++b) {
      if (geo.terrain && kzero<DIM>(a, b)) continue;
      const int c = comp_of<DIM>(b);
      utb[a] += K[a][b] * P.ub[c];
      utp[a] += K[a][b] * P.up[c];
      mtp[a] += K[a][b] * p5[1 + c];
    }
  }
  float r[9];
#pragma unroll
  for (int fld = 0; fld < 9; ++fld) {
    if (DIM == 2 && fld == 6) {
      r[fld] = 0.f;
      continue;
    }
    const int pb = DIM == 3 ? fld - 5 : (fld == 5 ? 0 : 1);
    const int msk = (fld >= 5 && fld <= 7) ? amask_of<DIM>(geo.terrain, pb) : (1 << DIM) - 1;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      if (!((msk >> a) & 1)) continue;
      float v;
      if (fld == 0) v = mtp[a];
      else if (fld <= 3) v = b5[fld] * utp[a] + p5[fld] * (utb[a] + utp[a]);
      else if (fld == 4) v = P.rkb * utp[a] + P.rkp * (utb[a] + utp[a]);
      else if (fld <= 7) v = P.pp * K[a][pb];
      else v = hb * utp[a] + hp * (utb[a] + utp[a]);
      sm[le][a][i] = v;
    }
    __syncthreads();
    r[fld] = contract<float, DIM, N>(tb, sm[le], i, idx, msk);
    __syncthreads();
  }
  if (!active) return;
  lift<float, DIM, N, 9>(tb, slot, S, e, idx, r);
#pragma unroll
  for (int fld = 0; fld < 5; ++fld) fns[fld * Nn + node] = iM * r[fld];
  // sources are linear: -rho' g k - f rho k x u' ... as (f m'_y, -f m'_x, -g rho'), -g m'_z
  const float ff = fcell32 ? __ldg(fcell32 + e) : f;
  fs[0 * Nn + node] = iM * r[5] + ff * p5[2];
  fs[1 * Nn + node] = iM * r[6] - ff * p5[1];
  fs[2 * Nn + node] = iM * r[7] - g * p5[0];
  fs[3 * Nn + node] = iM * r[8] - g * p5[3];
}

}  // namespace dg

namespace dg {

// background rates F(qb) in FP64, kept with the physics they were made for
static int bg_rates(dg_mesh* m, const PhysK& ph, cudaStream_t st) {
  int rc = DG_ERR_UNSUPPORTED;
  double* F = m->bgF.as<double>();
  DG_DISPATCH(m, rc = (Engine<double, D_, N_>::explicit_rates(m, ph, m->bg.as<double>(), F, F + 5 * m->N, st)));
  if (rc != DG_OK) return rc;
  m->bg_gamma = ph.gamma;
  m->bg_g = ph.g;
  m->bg_f = ph.f;
  m->bg_lmin = ph.lambda_min;
  m->bg_fcell = ph.fcell;
  return DG_OK;
}

// face data of a background qb (device, FP64): FP32 copy, FP32 traces for
// the perturbation fluxes, FP64 jumps and lambdab at face points
template <int DIM, int N>
static int bg_faces(dg_mesh* m, const double* qb, double gamma, cudaStream_t st) {
  const int64_t n = m->N;
  Tables<double> tb = m->tab.t;
  Tables<float> tb32 = cast_tables<float>(m->tab.t);
  FaceTopo ft = topo(m);
  Fields<double> in;
  Fields<float> in32;
  for (int k = 0; k < 5; ++k) {
    in.f[k] = qb + k * n;
    in.scale[k] = 1;
    in32.f[k] = m->bg32.as<float>() + k * n;
    in32.scale[k] = 1;
  }
  DG_RUN(m, K_VEC, st, k_bg_cast<<<grid_for(5 * n, 256), 256, 0, st>>>(qb, m->bg32.as<float>(), 5 * n));
  DG_RUN(m, K_TRACE, st, k_trace<double, DIM, N, 5><<<trace_grid<DIM, N>(m->E), TraceShape<DIM, N>::THREADS, 0, st>>>(in, m->E, n, m->trc.as<double>(), m->S, tb));
  DG_RUN(m, K_FACE_EXPLICIT, st, k_bg_jumps<DIM, N><<<grid_for(m->nF, 128), 128, 0, st>>>(ft, m->trc.as<double>(), tb, gamma, m->bgjump.as<float>()));
  DG_RUN(m, K_TRACE, st, k_trace<float, DIM, N, 5><<<trace_grid<DIM, N>(m->E), TraceShape<DIM, N>::THREADS, 0, st>>>(in32, m->E, n, m->bgtr.as<float>(), m->S, tb32));
  DG_LAUNCH_CHECK("background faces");
  return DG_OK;
}

static int bg_buffers(dg_mesh* m) {
  int rc;
  const int64_t n = m->N;
  if ((rc = ensure_fp32_geometry(m)) != DG_OK) return rc;
  if ((rc = m->bg32.ensure(sizeof(float) * 5 * n)) != DG_OK) return rc;
  if ((rc = m->bgtr.ensure(sizeof(float) * 5 * m->S)) != DG_OK) return rc;
  if ((rc = m->bgjump.ensure(sizeof(float) * 7 * (m->nF > 0 ? m->nF : 1))) != DG_OK) return rc;
  if ((rc = m->trc.ensure(sizeof(double) * 5 * m->S)) != DG_OK) return rc;
  return DG_OK;
}

int set_background(dg_mesh* m, const PhysK& ph, const double* qb, cudaStream_t st) {
  int rc;
  const int64_t n = m->N;
  m->bg_set = false;
  if ((rc = bg_buffers(m)) != DG_OK) return rc;
  if ((rc = m->bg.ensure(sizeof(double) * 5 * n)) != DG_OK) return rc;
  if ((rc = m->bgF.ensure(sizeof(double) * 9 * n)) != DG_OK) return rc;
  DG_CUDA(cudaMemcpyAsync(m->bg.as<double>(), qb, sizeof(double) * 5 * n, cudaMemcpyDeviceToDevice, st));
  rc = DG_ERR_UNSUPPORTED;
  DG_DISPATCH(m, rc = (bg_faces<D_, N_>(m, m->bg.as<double>(), ph.gamma, st)));
  if (rc != DG_OK) return rc;
  if ((rc = bg_rates(m, ph, st)) != DG_OK) return rc;
  m->bg_set = true;
  return DG_OK;
}

// F(q) = F(qb) + F' with F' in FP32 from q' = q - qb; fb_ns (5 x N) and
// fb_s (4 x N) hold F(qb), the face data of qb are in bg32/bgtr/bgjump
template <int DIM, int N>
static int explicit_pert_impl(dg_mesh* m, const PhysK& ph, const double* q, const double* qb,
                              const double* fb_ns, const double* fb_s, double* fns, double* fs,
                              cudaStream_t st) {
  using CS = CellShape<DIM, N>;
  const int64_t n = m->N;
  int rc;
  if ((rc = m->trc.ensure(sizeof(double) * 5 * m->S)) != DG_OK) return rc;
  if ((rc = m->slot.ensure(sizeof(double) * 9 * m->S)) != DG_OK) return rc;
  if ((rc = m->hbuf.ensure(sizeof(double) * 9 * (m->nH > 0 ? m->nH : 1))) != DG_OK) return rc;
  if ((rc = m->pert32.ensure(sizeof(float) * (14 * n + m->E))) != DG_OK) return rc;
  float* qp = m->pert32.as<float>();
  float* Fp = qp + 5 * n;           // 5 n non-stiff then 4 n stiff
  float* fc32 = Fp + 9 * n;
  float* trp = reinterpret_cast<float*>(m->trc.p);
  float* slot = reinterpret_cast<float*>(m->slot.p);
  float* hbuf = reinterpret_cast<float*>(m->hbuf.p);
  Tables<float> tb = cast_tables<float>(m->tab.t);
  FaceTopo ft = topo(m);
  const unsigned g5 = grid_for(5 * n, 256);
  DG_RUN(m, K_VEC, st, k_perturbation<<<g5, 256, 0, st>>>(q, qb, 5 * n, qp));
  if (ph.fcell) DG_RUN(m, K_VEC, st, k_bg_cast<<<grid_for(m->E, 256), 256, 0, st>>>(ph.fcell, fc32, m->E));
  Fields<float> in;
  for (int k = 0; k < 5; ++k) {
    in.f[k] = qp + k * n;
    in.scale[k] = 1;
  }
  DG_RUN(m, K_TRACE, st, k_trace<float, DIM, N, 5><<<trace_grid<DIM, N>(m->E), TraceShape<DIM, N>::THREADS, 0, st>>>(in, m->E, n, trp, m->S, tb));
  DG_RUN(m, K_FACE_EXPLICIT, st,
         k_face_explicit_pert<DIM, N><<<grid_for(m->nF, 128), 128, 0, st>>>(
             ft, trp, m->bgtr.as<float>(), m->bgjump.as<float>(), slot, hbuf, tb, (float)ph.gamma,
             (float)ph.lambda_min));
  if (m->nHC > 0)
    DG_RUN(m, K_HANG_GATHER, st, k_hang_gather<float, DIM, N, 9><<<grid_for(m->nHC * CS::NFP, 128), 128, 0, st>>>(ft, hbuf, slot, tb));
  DG_RUN(m, K_VOL_EXPLICIT, st,
         k_volume_explicit_pert<DIM, N><<<grid_for(m->E, CS::EPB), CS::THREADS, 0, st>>>(
             qp, m->bg32.as<float>(), cell_geo<float>(m), slot, m->E, m->S, tb, (float)ph.gamma,
             (float)ph.g, (float)ph.f, ph.fcell ? fc32 : nullptr, Fp, Fp + 5 * n));
  DG_RUN(m, K_VEC, st, k_add_rates<<<g5, 256, 0, st>>>(fb_ns, Fp, 5 * n, fns));
  DG_RUN(m, K_VEC, st, k_add_rates<<<grid_for(4 * n, 256), 256, 0, st>>>(fb_s, Fp + 5 * n, 4 * n, fs));
  DG_LAUNCH_CHECK("explicit operator (perturbation form)");
  return DG_OK;
}

int explicit_mixed(dg_mesh* m, const PhysK& ph, const double* q, double* fns, double* fs, cudaStream_t st) {
  int rc;
  if (ph.gamma != m->bg_gamma || ph.g != m->bg_g || ph.f != m->bg_f || ph.fcell != m->bg_fcell ||
      ph.lambda_min != m->bg_lmin)
    if ((rc = bg_rates(m, ph, st)) != DG_OK) return rc;   // background rates for these physics
  const double* Fb = m->bgF.as<double>();
  rc = DG_ERR_UNSUPPORTED;
  DG_DISPATCH(m, rc = (explicit_pert_impl<D_, N_>(m, ph, q, m->bg.as<double>(), Fb, Fb + 5 * m->N, fns, fs, st)));
  return rc;
}

int increment_begin(dg_mesh* m, double gamma, const double* q0, cudaStream_t st) {
  int rc;
  if ((rc = bg_buffers(m)) != DG_OK) return rc;
  rc = DG_ERR_UNSUPPORTED;
  DG_DISPATCH(m, rc = (bg_faces<D_, N_>(m, q0, gamma, st)));
  return rc;
}

int explicit_increment(dg_mesh* m, const PhysK& ph, const double* q, const double* q0, const double* f0_ns,
                       const double* f0_s, double* fns, double* fs, cudaStream_t st) {
  int rc = DG_ERR_UNSUPPORTED;
  DG_DISPATCH(m, rc = (explicit_pert_impl<D_, N_>(m, ph, q, q0, f0_ns, f0_s, fns, fs, st)));
  return rc;
}

}  // namespace dg

using namespace dg;

extern "C" int dg_mesh_set_background(dg_ctx* ctx, dg_mesh* mesh, const dg_phys* ph, const double* q_bg,
                                      void* stream) {
  if (!ctx || !mesh || !ph || !q_bg) {
    set_error("dg_mesh_set_background: NULL argument");
    return DG_ERR_ARG;
  }
  if (!(ph->gamma > 1.0)) {
    set_error("dg_mesh_set_background: gamma must be > 1");
    return DG_ERR_ARG;
  }
  if (mesh->gll || mesh->nFar > 0) {
    set_error("dg_mesh_set_background: not implemented for Gauss-Lobatto nodes or far-field faces");
    return DG_ERR_UNSUPPORTED;
  }
  PhysK k{ph->gamma, ph->g, ph->f, ph->f_cell, ph->lambda_min};
  return set_background(mesh, k, q_bg, (cudaStream_t)stream);
}
