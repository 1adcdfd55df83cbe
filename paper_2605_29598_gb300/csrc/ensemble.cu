// Ensembles of independent instances stepped together.
//
// Instances that share (dim, degree) are merged into one mesh (a disjoint
// union of their cells and face lists, cell indices offset), so every
// kernel of a step covers all of them in one launch; the Coriolis parameter
// is carried per cell.  Each group is advanced by imex_ark2_step, with one
// GMRES / Picard iteration for the whole group (a block-diagonal system
// whose stopping tests use norms over the group).
#include <cmath>
#include <map>
#include <string>
#include <thread>
#include <vector>

#include "engine.cuh"

struct dg_ensemble {
  dg_ctx* ctx = nullptr;
  struct Group {
    int dim = 0, degree = 0;
    dg_mesh* mesh = nullptr;
    double* f_cell = nullptr;     // device, one per merged cell
    double* q = nullptr;          // device, 5 x N merged state
    std::vector<int> members;     // instance ids
    cudaStream_t stream = nullptr;  // groups step concurrently, one stream each
    cudaEvent_t done = nullptr;
  };
  cudaEvent_t start = nullptr;
  std::vector<Group> groups;
  MultiGraph* graph = nullptr;   // all groups' steps as one CUDA graph (opts.graph)
  struct Inst {
    int group = -1;
    int64_t cell_off = 0, n_elem = 0, n_nodes = 0;
  };
  std::vector<Inst> inst;
};

using namespace dg;

extern "C" {

void dg_ensemble_destroy(dg_ensemble* e) {
  if (!e) return;
  for (auto& g : e->groups) {
    dg_mesh_destroy(g.mesh);
    cudaFree(g.f_cell);
    cudaFree(g.q);
    if (g.stream) cudaStreamDestroy(g.stream);
    if (g.done) cudaEventDestroy(g.done);
  }
  if (e->start) cudaEventDestroy(e->start);
  multi_graph_release(e->graph);
  delete e;
}

int dg_ensemble_create(dg_ctx* ctx, const dg_mesh_desc* descs, const double* f_inst, int n,
                       dg_ensemble** out) {
  if (!ctx || !descs || !f_inst || n <= 0 || !out) {
    set_error("dg_ensemble_create: NULL argument or n <= 0");
    return DG_ERR_ARG;
  }
  *out = nullptr;
  dg_ensemble* ens = new dg_ensemble;
  ens->ctx = ctx;
  ens->inst.resize(n);
  std::map<std::pair<int, int>, int> gid;
  for (int i = 0; i < n; ++i) {
    const dg_mesh_desc& d = descs[i];
    if (d.node_set != DG_NODES_GL) {
      dg_ensemble_destroy(ens);
      set_error("dg_ensemble_create: instance %d: ensembles take Gauss-Legendre nodes only", i);
      return DG_ERR_UNSUPPORTED;
    }
    for (int64_t k = 0; k < d.n_bdry && d.bdry_faces; ++k)
      if (d.bdry_faces[3 * k + 2] == DG_BC_FARFIELD) {
        dg_ensemble_destroy(ens);
        set_error("dg_ensemble_create: instance %d: ensembles take slip walls only", i);
        return DG_ERR_UNSUPPORTED;
      }
    if ((d.dim != 2 && d.dim != 3) || d.n_elem <= 0) {
      dg_ensemble_destroy(ens);
      set_error("dg_ensemble_create: instance %d has an invalid mesh description", i);
      return DG_ERR_ARG;
    }
    auto key = std::make_pair(d.dim, d.degree);
    if (!gid.count(key)) {
      gid[key] = (int)ens->groups.size();
      ens->groups.push_back({});
      ens->groups.back().dim = d.dim;
      ens->groups.back().degree = d.degree;
    }
    ens->inst[i].group = gid[key];
    ens->groups[gid[key]].members.push_back(i);
  }
  for (auto& g : ens->groups) {
    std::vector<double> verts;
    std::vector<int64_t> inf, hf, bf;
    std::vector<double> fc;
    int64_t off = 0;
    const int nv = g.dim << g.dim;
    for (int i : g.members) {
      const dg_mesh_desc& d = descs[i];
      if (d.node_set != descs[g.members[0]].node_set || !d.vertices) {
        dg_ensemble_destroy(ens);
        set_error("dg_ensemble_create: instance %d: mixed node sets or NULL vertices", i);
        return DG_ERR_ARG;
      }
      ens->inst[i].cell_off = off;
      ens->inst[i].n_elem = d.n_elem;
      verts.insert(verts.end(), d.vertices, d.vertices + d.n_elem * nv);
      for (int64_t k = 0; k < d.n_int; ++k) {
        const int64_t* r = d.int_faces + 4 * k;
        inf.insert(inf.end(), {r[0] + off, r[1], r[2] + off, r[3]});
      }
      for (int64_t k = 0; k < d.n_hang; ++k) {
        const int64_t* r = d.hang_faces + 5 * k;
        hf.insert(hf.end(), {r[0] + off, r[1], r[2] + off, r[3], r[4]});
      }
      for (int64_t k = 0; k < d.n_bdry; ++k) {
        const int64_t* r = d.bdry_faces + 3 * k;
        bf.insert(bf.end(), {r[0] + off, r[1], r[2]});
      }
      fc.insert(fc.end(), d.n_elem, f_inst[i]);
      off += d.n_elem;
    }
    dg_mesh_desc md = descs[g.members[0]];
    md.n_elem = off;
    md.vertices = verts.data();
    md.n_int = (int64_t)inf.size() / 4;
    md.int_faces = inf.data();
    md.n_hang = (int64_t)hf.size() / 5;
    md.hang_faces = hf.data();
    md.n_bdry = (int64_t)bf.size() / 3;
    md.bdry_faces = bf.data();
    int rc = dg_mesh_create(ctx, &md, &g.mesh);
    if (rc != DG_OK) {
      dg_ensemble_destroy(ens);
      return rc;
    }
    cudaError_t e = cudaMalloc(&g.f_cell, sizeof(double) * off);
    if (e == cudaSuccess) e = cudaMemcpy(g.f_cell, fc.data(), sizeof(double) * off, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&g.q, sizeof(double) * 5 * g.mesh->N);
    if (e == cudaSuccess) e = cudaMemset(g.q, 0, sizeof(double) * 5 * g.mesh->N);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&g.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g.done, cudaEventDisableTiming);
    if (e != cudaSuccess) {
      dg_ensemble_destroy(ens);
      return cuda_fail(e, "dg_ensemble_create");
    }
    for (int i : g.members) ens->inst[i].n_nodes = ens->inst[i].n_elem * g.mesh->Np;
    // degree-specialised tile schedule of this group, picked by timing
    rc = dg_mesh_autotune(ctx, g.mesh, DG_MIXED, nullptr);
    if (rc != DG_OK) {
      dg_ensemble_destroy(ens);
      return rc;
    }
  }
  {
    cudaError_t e = cudaEventCreateWithFlags(&ens->start, cudaEventDisableTiming);
    if (e != cudaSuccess) {
      dg_ensemble_destroy(ens);
      return cuda_fail(e, "dg_ensemble_create");
    }
  }
  *out = ens;
  return DG_OK;
}

int dg_ensemble_info(const dg_ensemble* e, int* n_groups, int64_t* total_nodes) {
  if (!e) {
    set_error("dg_ensemble_info: NULL ensemble");
    return DG_ERR_ARG;
  }
  int64_t t = 0;
  for (auto& g : e->groups) t += g.mesh->N;
  if (n_groups) *n_groups = (int)e->groups.size();
  if (total_nodes) *total_nodes = t;
  return DG_OK;
}

int dg_ensemble_instance_nodes(const dg_ensemble* e, int i, int64_t* n_nodes) {
  if (!e || i < 0 || i >= (int)e->inst.size() || !n_nodes) {
    set_error("dg_ensemble_instance_nodes: bad argument");
    return DG_ERR_ARG;
  }
  *n_nodes = e->inst[i].n_nodes;
  return DG_OK;
}

// copy instance i's state (5 x N_i, device) into or out of the merged state
static int copy_instance(dg_ensemble* e, int i, double* q, bool to_merged, cudaStream_t st) {
  if (!e || i < 0 || i >= (int)e->inst.size() || !q) {
    set_error("dg_ensemble_%s_state: bad argument", to_merged ? "set" : "get");
    return DG_ERR_ARG;
  }
  const auto& in = e->inst[i];
  const auto& g = e->groups[in.group];
  const int64_t Ng = g.mesh->N, Np = g.mesh->Np;
  for (int k = 0; k < 5; ++k) {
    double* merged = g.q + k * Ng + in.cell_off * Np;
    double* mine = q + k * in.n_nodes;
    DG_CUDA(cudaMemcpyAsync(to_merged ? merged : mine, to_merged ? mine : merged,
                            sizeof(double) * in.n_nodes, cudaMemcpyDeviceToDevice, st));
  }
  return DG_OK;
}

int dg_ensemble_set_state(dg_ensemble* e, int i, const double* q, void* stream) {
  return copy_instance(e, i, const_cast<double*>(q), true, (cudaStream_t)stream);
}

int dg_ensemble_get_state(dg_ensemble* e, int i, double* q, void* stream) {
  return copy_instance(e, i, q, false, (cudaStream_t)stream);
}

int dg_ensemble_step(dg_ensemble* e, const dg_phys* ph, const double* dt_inst, const dg_step_opts* opts,
                     dg_step_info* info, void* stream) {
  if (!e || !ph || !dt_inst || !opts) {
    set_error("dg_ensemble_step: NULL argument");
    return DG_ERR_ARG;
  }
  for (auto& g : e->groups)
    for (int i : g.members)
      if (dt_inst[i] != dt_inst[g.members[0]]) {
        set_error("dg_ensemble_step: instances %d and %d share (dim, degree) but not dt", g.members[0], i);
        return DG_ERR_ARG;
      }
  cudaStream_t caller = (cudaStream_t)stream;
  if (opts->graph) {
    // every group's step as a parallel branch of one graph: one launch
    const size_t ng = e->groups.size();
    std::vector<dg_mesh*> meshes(ng);
    std::vector<dg_phys> phs(ng, *ph);
    std::vector<double*> qs(ng);
    std::vector<double> dts(ng);
    std::vector<dg_step_info> infos(ng);
    for (size_t k = 0; k < ng; ++k) {
      meshes[k] = e->groups[k].mesh;
      phs[k].f_cell = e->groups[k].f_cell;
      qs[k] = e->groups[k].q;
      dts[k] = dt_inst[e->groups[k].members[0]];
    }
    int rc = multi_step_graph((int)ng, meshes.data(), phs.data(), qs.data(), dts.data(), opts, infos.data(),
                              &e->graph, caller);
    if (rc != DG_OK) return rc;
    dg_step_info total{};
    for (const auto& gi : infos) {
      for (int l = 0; l < 3; ++l) total.picard_iters[l] = std::max(total.picard_iters[l], gi.picard_iters[l]);
      total.gmres_iters_total += gi.gmres_iters_total;
      total.max_relres = std::max(total.max_relres, gi.max_relres);
      total.refinements_total += gi.refinements_total;
    }
    if (info) *info = total;
    return DG_OK;
  }
  // Each group steps on its own stream from its own host thread, so groups
  // overlap on the GPU (their GMRES loops synchronise only their stream).
  // The caller's stream orders before and after all of them.
  DG_CUDA(cudaEventRecord(e->start, caller));
  const size_t ng = e->groups.size();
  std::vector<int> rcs(ng, DG_OK);
  std::vector<dg_step_info> infos(ng);
  std::vector<std::string> errs(ng);
  std::vector<std::thread> workers;
  const int device = e->ctx->device;
  for (size_t k = 0; k < ng; ++k) {
    workers.emplace_back([&, k] {
      auto& g = e->groups[k];
      cudaSetDevice(device);
      cudaError_t ce = cudaStreamWaitEvent(g.stream, e->start, 0);
      if (ce != cudaSuccess) {
        rcs[k] = DG_ERR_CUDA;
        errs[k] = cudaGetErrorString(ce);
        return;
      }
      dg_phys pg = *ph;
      pg.f_cell = g.f_cell;
      rcs[k] = imex_ark2_step(e->ctx, g.mesh, &pg, g.q, dt_inst[g.members[0]], opts, &infos[k], g.stream);
      if (rcs[k] != DG_OK) errs[k] = dg_last_error();
      cudaEventRecord(g.done, g.stream);
    });
  }
  for (auto& w : workers) w.join();
  for (auto& g : e->groups) DG_CUDA(cudaStreamWaitEvent(caller, g.done, 0));
  dg_step_info total{};
  for (size_t k = 0; k < ng; ++k) {
    if (rcs[k] != DG_OK) {
      set_error("dg_ensemble_step: group %d: %s", (int)k, errs[k].c_str());
      return rcs[k];
    }
    const dg_step_info& gi = infos[k];
    for (int l = 0; l < 3; ++l) total.picard_iters[l] = std::max(total.picard_iters[l], gi.picard_iters[l]);
    total.gmres_iters_total += gi.gmres_iters_total;
    total.max_relres = std::max(total.max_relres, gi.max_relres);
    total.refinements_total += gi.refinements_total;
  }
  if (info) *info = total;
  return DG_OK;
}

}  // extern "C"
