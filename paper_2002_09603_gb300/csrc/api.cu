// C ABI of libmhfp: argument validation, handle life cycle, dispatch.
#include "common.cuh"

#include <chrono>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

namespace mhfp {

long long g_launches = 0;
thread_local LaneCfg g_lane;

void* dalloc(Ctx& c, size_t bytes) {
  void* p = nullptr;
  if (bytes == 0) bytes = 8;
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    throw Error{MHFP_ERR_OOM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed"};
  }
  c.allocs.push_back(p);
  return p;
}

void dfree_all(Ctx& c) {
  for (void* p : c.allocs) cudaFree(p);
  c.allocs.clear();
}

void timing_begin(Ctx& c, int cls) {
  if (c.suppress_events) return;
  if (c.timing.capturing) {
    // inside a graph capture: an external event-record node that records on
    // every replay; the pair is read after each replay
    TimedPair t{cls, nullptr, nullptr, 0.0, false};
    MHFP_CUDA(cudaEventCreate(&t.start));
    MHFP_CUDA(cudaEventCreate(&t.stop));
    MHFP_CUDA(cudaEventRecordWithFlags(t.start, c.stream, cudaEventRecordExternal));
    c.timing.capture_list->push_back(t);
    return;
  }
  if (!c.timing.enabled) return;
  auto& v = c.timing.ev_start[cls];
  if (c.timing.used[cls] >= v.size()) {
    cudaEvent_t a, b;
    MHFP_CUDA(cudaEventCreate(&a));
    MHFP_CUDA(cudaEventCreate(&b));
    c.timing.ev_start[cls].push_back(a);
    c.timing.ev_stop[cls].push_back(b);
  }
  MHFP_CUDA(cudaEventRecord(c.timing.ev_start[cls][c.timing.used[cls]], c.stream));
}

static void harvest(Ctx& c, int cls) {
  MHFP_CUDA(cudaStreamSynchronize(c.stream));
  for (size_t i = 0; i < c.timing.used[cls]; ++i) {
    float ms = 0.f;
    MHFP_CUDA(cudaEventElapsedTime(&ms, c.timing.ev_start[cls][i], c.timing.ev_stop[cls][i]));
    c.timing.total_ms[cls] += ms;
  }
  c.timing.used[cls] = 0;
}

void timing_end(Ctx& c, int cls, double bytes) {
  if (c.suppress_events) return;
  if (c.timing.capturing) {
    // the innermost open pair of this class (classes nest)
    auto& list = *c.timing.capture_list;
    for (size_t i = list.size(); i-- > 0;) {
      TimedPair& t = list[i];
      if (t.cls != cls || t.closed) continue;
      t.bytes = bytes;
      t.closed = true;
      MHFP_CUDA(cudaEventRecordWithFlags(t.stop, c.stream, cudaEventRecordExternal));
      return;
    }
    throw Error{MHFP_ERR_STATE, "timing_end without timing_begin"};
  }
  if (!c.timing.enabled) return;
  MHFP_CUDA(cudaEventRecord(c.timing.ev_stop[cls][c.timing.used[cls]], c.stream));
  c.timing.used[cls]++;
  c.timing.launches[cls]++;
  c.timing.bytes[cls] += bytes;
  if (c.timing.used[cls] >= 4096) harvest(c, cls);
}

}  // namespace mhfp

using mhfp::Ctx;
using mhfp::Error;

struct mhfp_ctx {
  Ctx c;
};

namespace {

template <class F>
mhfp_status guarded(mhfp_handle h, F&& f) {
  if (!h) return MHFP_ERR_ARG;
  try {
    MHFP_CUDA(cudaSetDevice(h->c.device));
    f(h->c);
    h->c.err.clear();
    return MHFP_OK;
  } catch (const Error& e) {
    h->c.err = e.msg;
    return e.status;
  } catch (const std::bad_alloc&) {
    h->c.err = "host allocation failed";
    return MHFP_ERR_OOM;
  }
}

// which = 0: displacement; 1: interface pressure (C~_p with the mixed
// formulation); 2: the mixed formulation's A_qq level
std::vector<mhfp::Level>& hierarchy_of(Ctx& c, int which) {
  if (which == 0) return c.hu;
  if (c.opt.formulation == 1) return which == 1 ? c.hcp : c.hq;
  return c.hpi;
}

// the calls that only the hybridized system has
void hybrid_only(const Ctx& c) {
  if (c.opt.formulation == 1) throw Error{MHFP_ERR_STATE, "not available with the mixed formulation"};
}

template <class T>
T* upload(Ctx& c, const T* host, size_t n) {
  T* d = mhfp::dalloc_n<T>(c, n);
  MHFP_CUDA(cudaMemcpyAsync(d, host, n * sizeof(T), cudaMemcpyHostToDevice, c.stream));
  return d;
}

}  // namespace

extern "C" {

void mhfp_default_options(mhfp_options* o) {
  if (!o) return;
  o->restart = 50;
  o->maxit = 1000;
  o->cheb_degree = 2;
  o->cheb_ratio = 10.0;
  o->coarse_max = 125;
  o->power_iters = 15;
  o->precision = 0;
  o->graphs = 2;
  o->autotune = 1;
  o->reorth = 1;
  o->schedule = 0;
  o->fine_blocks = 0;
  o->near_kernel = 0;
  o->formulation = 0;
}

const char* mhfp_status_string(mhfp_status s) {
  switch (s) {
    case MHFP_OK: return "ok";
    case MHFP_ERR_ARG: return "invalid argument";
    case MHFP_ERR_MESH: return "invalid mesh";
    case MHFP_ERR_OOM: return "out of memory";
    case MHFP_ERR_CUDA: return "CUDA error";
    case MHFP_ERR_NOT_CONVERGED: return "not converged";
    case MHFP_ERR_NONFINITE: return "non-finite value";
    case MHFP_ERR_BREAKDOWN: return "Krylov breakdown";
    case MHFP_ERR_STATE: return "call out of order";
  }
  return "unknown status";
}

const char* mhfp_last_error(mhfp_handle h) { return h ? h->c.err.c_str() : "null handle"; }

mhfp_status mhfp_create(const mhfp_mesh* mesh, const mhfp_materials* mat, double dt, const double traction[3],
                        void* stream, mhfp_handle* out) {
  if (!out) return MHFP_ERR_ARG;
  *out = nullptr;
  if (!mesh || !mat || !mesh->coords || !mesh->node_fix || !mesh->face_bc) return MHFP_ERR_ARG;
  if (!mat->E || !mat->nu || !mat->biot || !mat->Seps || !mat->mu || !mat->kappa) return MHFP_ERR_ARG;
  if (mesh->nx < 1 || mesh->ny < 1 || mesh->nz < 1) return MHFP_ERR_ARG;
  if (!(dt > 0.0) || !std::isfinite(dt)) return MHFP_ERR_ARG;
  const long long nx = mesh->nx, ny = mesh->ny, nz = mesh->nz;
  const long long nT = nx * ny * nz;
  if (nT > (1LL << 30)) return MHFP_ERR_ARG;
  // host-side validation of the material fields
  for (long long t = 0; t < nT; ++t) {
    const double E = mat->E[t], nu = mat->nu[t], mu = mat->mu[t], S = mat->Seps[t], b = mat->biot[t];
    if (!(E > 0.0) || !(nu > -1.0 && nu < 0.5) || !(mu > 0.0) || !(S >= 0.0) || !std::isfinite(b))
      return MHFP_ERR_ARG;
    for (int q = 0; q < 3; ++q)
      if (!(mat->kappa[3 * t + q] > 0.0) || !std::isfinite(mat->kappa[3 * t + q])) return MHFP_ERR_ARG;
  }
  mhfp_ctx* h = new (std::nothrow) mhfp_ctx;
  if (!h) return MHFP_ERR_OOM;
  Ctx& c = h->c;
  mhfp_default_options(&c.opt);
  c.nx = mesh->nx; c.ny = mesh->ny; c.nz = mesh->nz;
  c.nN = (nx + 1) * (ny + 1) * (nz + 1);
  c.nT = nT;
  c.nFx = (nx + 1) * ny * nz;
  c.nFy = nx * (ny + 1) * nz;
  c.nF = c.nFx + c.nFy + nx * ny * (nz + 1);
  c.nU = 3 * c.nN;
  c.n = c.nU + c.nT + c.nF;
  c.dt = dt;
  for (int q = 0; q < 3; ++q) c.trac[q] = traction ? traction[q] : 0.0;
  c.stream = (cudaStream_t)stream;
  try {
    int dev = 0;
    MHFP_CUDA(cudaGetDevice(&dev));
    c.device = dev;
    MHFP_CUDA(cudaDeviceGetAttribute(&c.n_sm, cudaDevAttrMultiProcessorCount, dev));
    for (long long i = 0; i < 3 * c.nN; ++i)
      if (!std::isfinite(mesh->coords[i])) throw Error{MHFP_ERR_ARG, "non-finite node coordinate"};
    c.coords = upload(c, mesh->coords, 3 * c.nN);
    c.node_fix = upload(c, mesh->node_fix, c.nN);
    c.face_bc = upload(c, mesh->face_bc, c.nF);
    c.E = upload(c, mat->E, nT);
    c.nu = upload(c, mat->nu, nT);
    c.biot = upload(c, mat->biot, nT);
    c.Seps = upload(c, mat->Seps, nT);
    c.mu = upload(c, mat->mu, nT);
    c.kappa = upload(c, mat->kappa, 3 * nT);
    c.d_flag = mhfp::dalloc_n<int>(c, 4);
    MHFP_CUDA(cudaStreamSynchronize(c.stream));
  } catch (const Error& e) {
    mhfp::dfree_all(c);
    delete h;
    return e.status;
  }
  *out = h;
  return MHFP_OK;
}

mhfp_status mhfp_assemble_condense(mhfp_handle h) {
  return guarded(h, [](Ctx& c) {
    if (c.assembled) throw Error{MHFP_ERR_STATE, "already assembled"};
    mhfp::assemble_all(c);
    c.assembled = true;
  });
}

mhfp_status mhfp_setup_precond(mhfp_handle h, const mhfp_options* opt) {
  return guarded(h, [&](Ctx& c) {
    if (!c.assembled) throw Error{MHFP_ERR_STATE, "mhfp_assemble_condense must come first"};
    if (c.prepared) throw Error{MHFP_ERR_STATE, "preconditioner already set up"};
    if (opt) {
      if (opt->restart < 1 || opt->restart > 63 || opt->maxit < 1 || opt->cheb_degree < 0 || opt->cheb_degree > 8 ||
          (opt->cheb_degree == 0 && opt->autotune != 1) ||
          !(opt->cheb_ratio > 1.0) || opt->coarse_max < 1 || opt->coarse_max > 4096 || opt->power_iters < 1 ||
          (opt->precision != 0 && opt->precision != 1) || (opt->graphs < 0 || opt->graphs > 2) ||
          (opt->autotune != 0 && opt->autotune != 1) || (opt->reorth != 0 && opt->reorth != 1) ||
          (opt->schedule != 0 && opt->schedule != 1 && opt->schedule != 4 && opt->schedule != 8 &&
           opt->schedule != 16) ||
          (opt->fine_blocks != 0 && (opt->fine_blocks < 4 || opt->fine_blocks > 8)) ||
          (opt->near_kernel != 0 && opt->near_kernel != 1) ||
          (opt->formulation != 0 && opt->formulation != 1) || (opt->formulation == 1 && opt->precision != 0))
        throw Error{MHFP_ERR_ARG, "invalid options"};
      c.opt = *opt;
    }
    const bool tune_degree = c.opt.cheb_degree == 0;
    if (tune_degree) c.opt.cheb_degree = 2;  // the hierarchy's set-up timings use degree 2
    mhfp::build_preconditioner_blocks(c);
    if (c.opt.formulation == 1) {
      mhfp::build_mixed_blocks(c);
      mhfp::build_mixed_hierarchies(c);
    } else {
      mhfp::build_hierarchies(c);
    }
    if (c.opt.precision == 1) mhfp::make_fp32_blocks(c);
    MHFP_CUDA(cudaStreamSynchronize(c.stream));
    c.prepared = true;
    if (tune_degree) {
      try {
        mhfp::autotune_cheb_degree(c);
      } catch (...) {
        c.prepared = false;
        throw;
      }
      MHFP_CUDA(cudaStreamSynchronize(c.stream));
    }
  });
}

mhfp_status mhfp_build_rhs(mhfp_handle h, const double* d_x_prev, double load_scale, double* d_rhs) {
  return guarded(h, [&](Ctx& c) {
    if (!c.assembled) throw Error{MHFP_ERR_STATE, "mhfp_assemble_condense must come first"};
    if (!d_rhs || !std::isfinite(load_scale)) throw Error{MHFP_ERR_ARG, "bad rhs argument"};
    mhfp::build_rhs(c, d_x_prev, load_scale, d_rhs);
  });
}

mhfp_status mhfp_solve(mhfp_handle h, const double* d_rhs, double* d_x, double tol, mhfp_stats* stats) {
  return guarded(h, [&](Ctx& c) {
    if (!c.prepared) throw Error{MHFP_ERR_STATE, "mhfp_setup_precond must come first"};
    if (!d_rhs || !d_x || !(tol > 0.0) || !(tol < 1.0)) throw Error{MHFP_ERR_ARG, "bad solve argument"};
    mhfp::fgmres_solve(c, d_rhs, d_x, tol, stats);
  });
}

mhfp_status mhfp_apply_operator(mhfp_handle h, const double* d_x, double* d_y) {
  return guarded(h, [&](Ctx& c) {
    if (!c.assembled || !c.prepared) throw Error{MHFP_ERR_STATE, "operator needs assemble + setup"};
    if (!d_x || !d_y || d_x == d_y) throw Error{MHFP_ERR_ARG, "bad vectors"};
    mhfp::apply_operator(c, d_x, d_y, nullptr, nullptr);
  });
}

mhfp_status mhfp_apply_operator_ff(mhfp_handle h, const double* d_x, double* d_y) {
  return guarded(h, [&](Ctx& c) {
    if (!c.assembled || !c.prepared) throw Error{MHFP_ERR_STATE, "operator needs assemble + setup"};
    if (c.opt.precision != 1 || c.opt.formulation != 0 || !c.auu_h)
      throw Error{MHFP_ERR_STATE, "the float-float operator needs a precision = 1 set-up"};
    if (!d_x || !d_y || d_x == d_y) throw Error{MHFP_ERR_ARG, "bad vectors"};
    mhfp::narrow_to_f32(c, d_x, c.zf, c.n);
    mhfp::apply_operator_arnoldi(c, d_x, c.zf, d_y, nullptr, false);
  });
}

mhfp_status mhfp_apply_operator_t(mhfp_handle h, const double* d_x, double* d_y) {
  return guarded(h, [&](Ctx& c) {
    hybrid_only(c);
    if (!c.assembled || !c.prepared) throw Error{MHFP_ERR_STATE, "operator needs assemble + setup"};
    if (!d_x || !d_y || d_x == d_y) throw Error{MHFP_ERR_ARG, "bad vectors"};
    mhfp::apply_operator(c, d_x, d_y, nullptr, nullptr, true);
  });
}

mhfp_status mhfp_adjoint_solve(mhfp_handle h, const double* d_g, double* d_lambda, double tol, mhfp_stats* stats) {
  return guarded(h, [&](Ctx& c) {
    hybrid_only(c);
    if (!c.prepared) throw Error{MHFP_ERR_STATE, "mhfp_setup_precond must come first"};
    if (!d_g || !d_lambda || !(tol > 0.0) || !(tol < 1.0)) throw Error{MHFP_ERR_ARG, "bad adjoint argument"};
    mhfp::fgmres_solve(c, d_g, d_lambda, tol, stats, true);
  });
}

mhfp_status mhfp_grad_logk(mhfp_handle h, const double* d_lambda, const double* d_x, double* d_grad) {
  return guarded(h, [&](Ctx& c) {
    hybrid_only(c);
    if (!c.assembled) throw Error{MHFP_ERR_STATE, "mhfp_assemble_condense must come first"};
    if (!d_lambda || !d_x || !d_grad) throw Error{MHFP_ERR_ARG, "bad gradient argument"};
    mhfp::grad_logk(c, d_lambda, d_x, d_grad);
  });
}

mhfp_status mhfp_misfit(mhfp_handle h, const double* d_x, const double* d_uz_target, const double* d_p_target,
                        double inv_su2, double inv_sp2, double* d_J, double* d_g) {
  return guarded(h, [&](Ctx& c) {
    if (!c.assembled) throw Error{MHFP_ERR_STATE, "mhfp_assemble_condense must come first"};
    if (!d_x || !d_uz_target || !d_p_target || !d_J || !d_g || !std::isfinite(inv_su2) || !std::isfinite(inv_sp2))
      throw Error{MHFP_ERR_ARG, "bad misfit argument"};
    mhfp::ensure_workspace(c);
    mhfp::misfit(c, d_x, d_uz_target, d_p_target, inv_su2, inv_sp2, d_J, d_g, c.partials,
                 (long long)(c.opt.restart + 2) * c.npart);
  });
}

mhfp_status mhfp_adjoint_rhs(mhfp_handle h, const double* d_g, const double* d_lambda_next, double* d_rhs) {
  return guarded(h, [&](Ctx& c) {
    hybrid_only(c);
    if (!c.assembled) throw Error{MHFP_ERR_STATE, "mhfp_assemble_condense must come first"};
    if (!d_g || !d_rhs) throw Error{MHFP_ERR_ARG, "bad adjoint rhs argument"};
    mhfp::adjoint_rhs(c, d_g, d_lambda_next, d_rhs);
  });
}

mhfp_status mhfp_apply_precond_t(mhfp_handle h, const double* d_v, double* d_z) {
  return guarded(h, [&](Ctx& c) {
    hybrid_only(c);
    if (!c.prepared) throw Error{MHFP_ERR_STATE, "mhfp_setup_precond must come first"};
    if (!d_v || !d_z || d_v == d_z) throw Error{MHFP_ERR_ARG, "bad vectors"};
    mhfp::apply_precond(c, d_v, d_z, true);
  });
}

mhfp_status mhfp_apply_precond(mhfp_handle h, const double* d_v, double* d_z) {
  return guarded(h, [&](Ctx& c) {
    if (!c.prepared) throw Error{MHFP_ERR_STATE, "mhfp_setup_precond must come first"};
    if (!d_v || !d_z || d_v == d_z) throw Error{MHFP_ERR_ARG, "bad vectors"};
    mhfp::apply_precond(c, d_v, d_z);
  });
}

mhfp_status mhfp_vcycle(mhfp_handle h, int which, const double* d_b, double* d_x) {
  return guarded(h, [&](Ctx& c) {
    if (!c.prepared) throw Error{MHFP_ERR_STATE, "mhfp_setup_precond must come first"};
    if (which != 0 && which != 1) throw Error{MHFP_ERR_ARG, "which must be 0 or 1"};
    if (!d_b || !d_x || d_b == d_x) throw Error{MHFP_ERR_ARG, "bad vectors"};
    mhfp::vcycle_api(c, hierarchy_of(c, which), d_b, d_x);
  });
}

mhfp_status mhfp_level_apply(mhfp_handle h, int which, int level, const double* d_x, double* d_y) {
  return guarded(h, [&](Ctx& c) {
    if (!c.prepared) throw Error{MHFP_ERR_STATE, "mhfp_setup_precond must come first"};
    if (which != 0 && which != 1 && !(which == 2 && c.opt.formulation == 1))
      throw Error{MHFP_ERR_ARG, "which must be 0 or 1 (or 2 with the mixed formulation)"};
    auto& H = hierarchy_of(c, which);
    if (level < 0 || level >= (int)H.size()) throw Error{MHFP_ERR_ARG, "level out of range"};
    if (!d_x || !d_y || d_x == d_y) throw Error{MHFP_ERR_ARG, "bad vectors"};
    mhfp::level_apply(c, H, level, d_x, d_y);
  });
}

mhfp_status mhfp_hierarchy(mhfp_handle h, int which, mhfp_hierarchy_info* info) {
  return guarded(h, [&](Ctx& c) {
    if (!c.prepared) throw Error{MHFP_ERR_STATE, "mhfp_setup_precond must come first"};
    if ((which != 0 && which != 1 && !(which == 2 && c.opt.formulation == 1)) || !info)
      throw Error{MHFP_ERR_ARG, "bad argument"};
    auto& H = hierarchy_of(c, which);
    std::memset(info, 0, sizeof(*info));
    info->levels = (int)H.size();
    info->cheb_degree = c.opt.cheb_degree;
    for (size_t l = 0; l < H.size() && l < 8; ++l) {
      info->points[l] = H[l].npts;
      info->block[l] = H[l].bs;
      info->lmax[l] = H[l].dense_inv ? 0.0 : H[l].lmax;
      const bool lattice = !H[l].dense_inv && !H[l].faces;
      info->schedule[l] = !lattice ? 0 : (H[l].tpp ? H[l].tpp : mhfp::level_schedule(c, H, (int)l));
      info->sweep_us[l] = H[l].sweep_us;
    }
  });
}

mhfp_status mhfp_get_scalings(mhfp_handle h, double* d_btilde, double* d_ds) {
  return guarded(h, [&](Ctx& c) {
    if (!c.prepared) throw Error{MHFP_ERR_STATE, "mhfp_setup_precond must come first"};
    if (d_btilde)
      MHFP_CUDA(cudaMemcpyAsync(d_btilde, c.opt.formulation == 1 ? c.Cp + (size_t)12 * c.nT : c.btilde,
                                c.nT * sizeof(double), cudaMemcpyDeviceToDevice, c.stream));
    if (d_ds) MHFP_CUDA(cudaMemcpyAsync(d_ds, c.ds, c.n * sizeof(double), cudaMemcpyDeviceToDevice, c.stream));
  });
}

mhfp_status mhfp_sizes(mhfp_handle h, long long* n_u, long long* n_p, long long* n_pi) {
  if (!h) return MHFP_ERR_ARG;
  if (n_u) *n_u = h->c.nU;
  if (n_p) *n_p = h->c.nT;
  if (n_pi) *n_pi = h->c.nF;
  return MHFP_OK;
}

mhfp_status mhfp_timing(mhfp_handle h, int enable) {
  return guarded(h, [&](Ctx& c) {
    MHFP_CUDA(cudaStreamSynchronize(c.stream));
    for (int k = 0; k < mhfp::TIMING_CLASSES; ++k) {
      c.timing.used[k] = 0;
      if (enable) {
        c.timing.launches[k] = 0;
        c.timing.total_ms[k] = 0.0;
        c.timing.bytes[k] = 0.0;
      }
    }
    c.timing.enabled = enable != 0;
  });
}

mhfp_status mhfp_timing_read(mhfp_handle h, int kernel_class, long long* launches, double* total_ms,
                             double* bytes_per_launch) {
  return guarded(h, [&](Ctx& c) {
    if (kernel_class < 0 || kernel_class >= mhfp::TIMING_CLASSES)
      throw Error{MHFP_ERR_ARG, "kernel class out of range"};
    mhfp::harvest(c, kernel_class);
    if (launches) *launches = c.timing.launches[kernel_class];
    if (total_ms) *total_ms = c.timing.total_ms[kernel_class];
    if (bytes_per_launch)
      *bytes_per_launch = c.timing.launches[kernel_class] ? c.timing.bytes[kernel_class] / c.timing.launches[kernel_class] : 0.0;
  });
}

mhfp_status mhfp_update_logk(mhfp_handle h, const double* d_logk) {
  return guarded(h, [&](Ctx& c) {
    hybrid_only(c);
    if (!c.prepared) throw Error{MHFP_ERR_STATE, "mhfp_setup_precond must come first"};
    if (!d_logk) throw Error{MHFP_ERR_ARG, "bad log-permeability vector"};
    mhfp::update_logk_blocks(c, d_logk);  // validates before changing anything
    mhfp::invalidate_graphs(c);
    mhfp::rebuild_pi_hierarchy(c);
    if (c.opt.precision == 1) mhfp::make_fp32_blocks(c);
    MHFP_CUDA(cudaStreamSynchronize(c.stream));
  });
}

mhfp_status mhfp_residual_norm_noalloc(mhfp_handle h, const double* d_b, const double* d_x, double* d_out) {
  return guarded(h, [&](Ctx& c) {
    hybrid_only(c);
    if (!c.prepared) throw Error{MHFP_ERR_STATE, "mhfp_setup_precond must come first"};
    if (!d_b || !d_x || !d_out) throw Error{MHFP_ERR_ARG, "bad vectors"};
    mhfp::residual_norm_noalloc(c, d_b, d_x, d_out);
  });
}

mhfp_status mhfp_solve_batch(int count, const mhfp_handle* hs, const double* const* d_rhs, double* const* d_x,
                             double tol, mhfp_stats* stats, mhfp_status* statuses) {
  if (count < 0 || (count > 0 && (!hs || !d_rhs || !d_x))) return MHFP_ERR_ARG;
  if (!(tol > 0.0) || !(tol < 1.0)) return MHFP_ERR_ARG;
  std::vector<mhfp::FgState> st(count);
  std::vector<mhfp_status> code(count, MHFP_OK);
  std::vector<char> active(count, 0);
  auto fail = [&](int i, mhfp_status s, const std::string& msg) {
    code[i] = s;
    active[i] = 0;
    if (hs[i]) hs[i]->c.err = msg;
  };
  for (int i = 0; i < count; ++i) {
    if (!hs[i] || !d_rhs[i] || !d_x[i]) { code[i] = MHFP_ERR_ARG; continue; }
    Ctx& c = hs[i]->c;
    try {
      MHFP_CUDA(cudaSetDevice(c.device));
      if (!c.prepared) throw Error{MHFP_ERR_STATE, "mhfp_setup_precond must come first"};
      if (!(c.opt.graphs == 2 && !c.timing.enabled)) mhfp::fgmres_begin(c, st[i], d_rhs[i], d_x[i], tol, false);
      active[i] = 1;
    } catch (const Error& e) {
      fail(i, e.status, e.msg);
    }
  }
  // device-driven solves: one graph launch per handle, all queued before any
  // is waited for
  std::vector<char> dev(count, 0);
  for (int i = 0; i < count; ++i) {
    if (!active[i]) continue;
    Ctx& c = hs[i]->c;
    if (c.opt.graphs != 2 || c.timing.enabled) continue;
    try {
      MHFP_CUDA(cudaSetDevice(c.device));
      st[i] = mhfp::FgState{};
      mhfp::solve_device_graph_launch(c, d_rhs[i], tol, false);
      dev[i] = 1;
    } catch (const Error& e) {
      fail(i, e.status, e.msg);
    }
  }
  for (int i = 0; i < count; ++i) {
    if (!dev[i]) continue;
    Ctx& c = hs[i]->c;
    try {
      MHFP_CUDA(cudaSetDevice(c.device));
      mhfp::solve_device_graph_finish(c, d_x[i], &st[i].stats);
      active[i] = 0;
    } catch (const Error& e) {
      fail(i, e.status, e.msg);
    }
  }
  // every round: drain each handle's stream and queue its next piece of
  // work; handles on distinct streams run concurrently on the device
  bool any = true;
  while (any) {
    any = false;
    for (int i = 0; i < count; ++i) {
      if (!active[i]) continue;
      Ctx& c = hs[i]->c;
      try {
        MHFP_CUDA(cudaSetDevice(c.device));
        MHFP_CUDA(cudaStreamSynchronize(c.stream));
        mhfp::fgmres_advance(c, st[i]);
        if (st[i].phase == mhfp::FgState::DONE) active[i] = 0;
      } catch (const Error& e) {
        fail(i, e.status, e.msg);
      }
      any = any || active[i];
    }
  }
  mhfp_status first = MHFP_OK;
  for (int i = 0; i < count; ++i) {
    if (stats) stats[i] = st[i].stats;
    if (statuses) statuses[i] = code[i];
    if (first == MHFP_OK && code[i] != MHFP_OK) first = code[i];
  }
  return first;
}

struct mhfp_batch_s {
  std::vector<mhfp_handle> hs;
  std::vector<int> gen;
  int device = 0;
  mhfp::BatchGraph g;
};

mhfp_status mhfp_batch_create(int count, const mhfp_handle* hs, const double* const* d_rhs, double* const* d_x,
                              double tol, mhfp_batch* out) {
  return mhfp_batch_create_lanes(count, hs, d_rhs, d_x, tol, 1, out);
}

mhfp_status mhfp_batch_create_lanes(int count, const mhfp_handle* hs, const double* const* d_rhs,
                                    double* const* d_x, double tol, int max_lanes, mhfp_batch* out) {
  if (!out) return MHFP_ERR_ARG;
  *out = nullptr;
  if (count < 1 || !hs || !d_rhs || !d_x || !(tol > 0.0) || !(tol < 1.0)) return MHFP_ERR_ARG;
  if (max_lanes < 1 || max_lanes > MHFP_MAX_LANES) return MHFP_ERR_ARG;
  for (int i = 0; i < count; ++i) {
    if (!hs[i] || !d_rhs[i] || !d_x[i]) return MHFP_ERR_ARG;
    if (!hs[i]->c.prepared) return MHFP_ERR_STATE;
    if (hs[i]->c.device != hs[0]->c.device) return MHFP_ERR_ARG;
    if (hs[i]->c.timing.enabled) return MHFP_ERR_STATE;
  }
  mhfp_batch b = new (std::nothrow) mhfp_batch_s;
  if (!b) return MHFP_ERR_OOM;
  b->device = hs[0]->c.device;
  std::vector<Ctx*> cs;
  std::vector<const double*> r;
  std::vector<double*> x;
  for (int i = 0; i < count; ++i) {
    b->hs.push_back(hs[i]);
    b->gen.push_back(hs[i]->c.graph_gen);
    cs.push_back(&hs[i]->c);
    r.push_back(d_rhs[i]);
    x.push_back(d_x[i]);
  }
  try {
    MHFP_CUDA(cudaSetDevice(b->device));
    for (Ctx* c : cs) MHFP_CUDA(cudaStreamSynchronize(c->stream));
    mhfp::build_batch_graph(b->g, cs, r, x, tol, max_lanes);
  } catch (const Error& e) {
    hs[0]->c.err = e.msg;
    mhfp::destroy_batch_graph(b->g);
    delete b;
    return e.status;
  }
  *out = b;
  return MHFP_OK;
}

mhfp_status mhfp_batch_run(mhfp_batch b, void* stream, mhfp_stats* stats, mhfp_status* statuses) {
  if (!b) return MHFP_ERR_ARG;
  const int count = (int)b->hs.size();
  for (int i = 0; i < count; ++i)
    if (b->hs[i]->c.graph_gen != b->gen[i]) {
      b->hs[i]->c.err = "a handle of the batch changed (mhfp_update_logk); create the batch again";
      return MHFP_ERR_STATE;
    }
  const auto t0 = std::chrono::steady_clock::now();
  try {
    MHFP_CUDA(cudaSetDevice(b->device));
    for (mhfp_handle h : b->hs) MHFP_CUDA(cudaStreamSynchronize(h->c.stream));
    mhfp::run_batch_graph(b->g, (cudaStream_t)stream);
  } catch (const Error& e) {
    b->hs[0]->c.err = e.msg;
    return e.status;
  }
  const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  mhfp_status first = MHFP_OK;
  for (int i = 0; i < count; ++i) {
    const mhfp::DevCtl& h = b->g.host_ctl[i];
    mhfp_status code = MHFP_OK;
    if (h.status == (int)MHFP_ERR_NONFINITE) code = MHFP_ERR_NONFINITE;
    else if (!h.converged) code = MHFP_ERR_NOT_CONVERGED;
    if (stats) {
      mhfp_stats s{};
      s.iterations = h.total;
      s.restarts = h.cycles;
      s.converged = h.converged;
      s.rel_residual = h.est;
      s.true_rel_residual = h.true_rel;
      s.solve_ms = ms;
      stats[i] = s;
    }
    if (statuses) statuses[i] = code;
    if (first == MHFP_OK && code != MHFP_OK) first = code;
  }
  return first;
}

void mhfp_batch_destroy(mhfp_batch b) {
  if (!b) return;
  cudaSetDevice(b->device);
  mhfp::destroy_batch_graph(b->g);
  delete b;
}

long long mhfp_launch_count(void) { return mhfp::g_launches; }

void mhfp_destroy(mhfp_handle h) {
  if (!h) return;
  Ctx& c = h->c;
  cudaSetDevice(c.device);
  cudaStreamSynchronize(c.stream);
  for (int k = 0; k < mhfp::TIMING_CLASSES; ++k) {
    for (auto e : c.timing.ev_start[k]) cudaEventDestroy(e);
    for (auto e : c.timing.ev_stop[k]) cudaEventDestroy(e);
  }
  if (c.host_scal) cudaFreeHost(c.host_scal);
  for (int t = 0; t < 2; ++t)
    for (auto& g : c.graphs[t]) {
      if (g.exec) cudaGraphExecDestroy(g.exec);
      for (auto& p : g.timed) {
        cudaEventDestroy(p.start);
        cudaEventDestroy(p.stop);
      }
    }
  if (c.cap_stream) cudaStreamDestroy(c.cap_stream);
  for (int t = 0; t < 2; ++t)
    if (c.solve_exec[t]) cudaGraphExecDestroy(c.solve_exec[t]);
  if (c.host_ctl) cudaFreeHost(c.host_ctl);
  mhfp::dfree_all(c);
  delete h;
}

}  // extern "C"
