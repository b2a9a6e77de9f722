// C ABI entry points (declared in include/hz.h).  Every call catches internal
// failures and returns an hz_status; nothing throws across the boundary.
#include "hz_internal.h"

#include <chrono>
#include <cmath>
#include <cstring>

namespace hz {
size_t gmres_red_doubles(int m, int nr);
}

using namespace hz;

namespace {

thread_local std::string g_last_error;

// Fine level (finite differences, Eq. 40) and, for two-grid, the coarse FE
// level that carries the domain decomposition; then the slabs.
double spacing(const hz_params& p) { return p.h > 0 ? p.h : 1.0 / p.n[0]; }

size_t n_dof(const hz_params& p) {
  size_t n = 1;
  for (int l = 0; l < p.dim; ++l) n *= (size_t)(p.n[l] + 2 * p.w_out - 1);
  return n;
}

void build_levels(hz_handle* h, const double* m_dev) {
  const hz_params& p = h->p;
  const double hh = spacing(p);
  build_level_fd(h, h->fine, p.n, p.w_out, hh, m_dev, p.dim == 3, h->s2);
  if (p.two_grid) {
    build_level_fe(h, h->coarse, h->fine, p.n, p.w_out, hh, h->s2);
    h->sweep = &h->coarse;
  } else {
    h->sweep = &h->fine;
  }
  h->sweep->J = p.J;
  h->sweep->w = p.w_dd;
  build_slabs(h, *h->sweep, h->s2);
}

hz_status fail(hz_handle* h, hz_status st, const std::string& msg) {
  if (h) { h->err.st = st; h->err.msg = msg; }
  g_last_error = msg;
  return st;
}

template <typename F>
hz_status guarded(hz_handle* h, F&& body) {
  try {
    body();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(h, HZ_ECUDA, cudaGetErrorString(e));
    if (h) { h->err.st = HZ_OK; h->err.msg.clear(); }
    return HZ_OK;
  } catch (const Failure& f) {
    return fail(h, f.st, f.msg);
  } catch (const std::exception& e) {
    return fail(h, HZ_ECUDA, e.what());
  }
}

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

size_t prec_size(const hz_params& p) { return p.precision == HZ_MIXED ? sizeof(c64) : sizeof(c128); }

void release_work(hz_handle* h) {
  for (void** q : {&h->pr_r, &h->pr_u, &h->pr_u2, &h->pr_g, &h->pr_B1, &h->pr_B2, &h->pr_Bnx, &h->tg_u, &h->tg_r,
                   &h->tg_t}) {
    dfree(*q);
    *q = nullptr;
  }
  dfree(h->V); dfree(h->Z); dfree(h->W); dfree(h->R); dfree(h->red); dfree(h->hcol);
  h->V = h->Z = h->W = h->R = h->hcol = nullptr;
  h->red = nullptr;
}

void validate(const hz_params* p) {
  auto bad = [](const std::string& m) { throw Failure(HZ_EINVAL, m); };
  if (!p) bad("params is NULL");
  if (p->dim != 2 && p->dim != 3) bad("dim must be 2 or 3");
  for (int l = 0; l < p->dim; ++l) {
    if (p->n[l] < 4) bad("every n[l] must be >= 4");
    if (p->two_grid && (p->n[l] % 2 != 0))
      bad("two_grid needs an even number of interior cells on every axis");
  }
  if (!(p->h >= 0)) bad("h must be >= 0 (0: 1 / n[0])");
  if (p->w_out < 0) bad("w_out must be >= 0");
  if (!(p->omega > 0)) bad("omega must be > 0");
  if (p->J < 1) bad("J must be >= 1");
  if (p->sweep != HZ_SWEEP_UD && p->sweep != HZ_SWEEP_X && p->sweep != HZ_SWEEP_NX)
    bad("sweep must be HZ_SWEEP_UD, HZ_SWEEP_X or HZ_SWEEP_NX");
  if (p->sweep == HZ_SWEEP_X && (p->J % 2 != 0)) bad("the X-sweep needs an even J");
  if (p->sweep == HZ_SWEEP_NX && (p->n_cell < 1 || p->n_cell > (p->J + 1) / 2))
    bad("the NX-sweep needs 1 <= n_cell <= (J + 1) / 2");
  if (p->w_dd < 1) bad("w_dd must be >= 1");
  if (p->precision != HZ_PLAIN_FP64 && p->precision != HZ_MIXED) bad("bad precision");
  if (p->gmres_m < 1 || p->gmres_m > 200) bad("gmres_m must be in 1..200");
  if (p->max_iter < 1) bad("max_iter must be >= 1");
  if (!(p->tol > 0)) bad("tol must be > 0");
  if (!(p->c_pml >= 0)) bad("c_pml must be >= 0 (0: mean wave speed)");
  if (p->max_rhs < 1 || p->max_rhs > 64) bad("max_rhs must be in 1..64");
  if (p->two_grid && (p->nu < 0 || !(p->omega_jac > 0))) bad("bad smoother parameters");
  if (p->block_3d != 0 && p->block_3d != 64 && p->block_3d != 128 && p->block_3d != 256)
    bad("block_3d must be 0, 64, 128 or 256");
  if (p->boundary != HZ_BOUNDARY_PML && p->boundary != HZ_BOUNDARY_SPONGE)
    bad("boundary must be HZ_BOUNDARY_PML or HZ_BOUNDARY_SPONGE");
  if (p->boundary == HZ_BOUNDARY_SPONGE) {
    if (p->w_out < 1) bad("a sponge needs w_out >= 1");
    if (!(p->sponge_damping > 0 && p->sponge_damping < 1)) bad("sponge_damping must be in (0, 1)");
  }
  // slab columns of the level carrying the decomposition (the coarse grid of
  // a sponge keeps no layers: every cell is merged in pairs)
  int N = !p->two_grid ? p->n[0] + 2 * p->w_out - 1
          : p->boundary == HZ_BOUNDARY_SPONGE ? (p->n[0] + 2 * p->w_out) / 2 - 1
                                              : 2 * p->w_out + p->n[0] / 2 - 1;
  if (N / p->J < 4) bad("slabs too thin: fewer than 4 columns per slab");
}

}  // namespace

namespace hz {
hz_status run_guarded(hz_handle* h, const std::function<void()>& body) {
  return guarded(h, body);
}
}  // namespace hz

extern "C" {

const char* hz_status_string(hz_status s) {
  switch (s) {
    case HZ_OK: return "HZ_OK";
    case HZ_EINVAL: return "HZ_EINVAL";
    case HZ_ENOMEM: return "HZ_ENOMEM";
    case HZ_ECUDA: return "HZ_ECUDA";
    case HZ_ENOTFACTORED: return "HZ_ENOTFACTORED";
    case HZ_ENOTCONV: return "HZ_ENOTCONV";
    case HZ_ETIMEOUT: return "HZ_ETIMEOUT";
    case HZ_EINACCURATE: return "HZ_EINACCURATE";
  }
  return "HZ_UNKNOWN";
}

const char* hz_last_error(const hz_handle* h) {
  if (h) return h->err.msg.c_str();
  return g_last_error.c_str();
}

hz_status hz_setup(const hz_params* p, const double* m_dev, hz_handle** out) {
  if (!out) return fail(nullptr, HZ_EINVAL, "out is NULL");
  *out = nullptr;
  hz_handle* h = new hz_handle();
  hz_status st = guarded(h, [&] {
    validate(p);
    if (!m_dev) throw Failure(HZ_EINVAL, "m_dev is NULL");
    h->p = *p;
    double t0 = now_s();
    HZ_CU(cudaGetDevice(&h->dev));
    HZ_CU(cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->dev));
    HZ_CU(cudaStreamCreateWithFlags(&h->s2, cudaStreamNonBlocking));
    HZ_CU(cudaEventCreateWithFlags(&h->evA, cudaEventDisableTiming));
    HZ_CU(cudaEventCreateWithFlags(&h->evB, cudaEventDisableTiming));
    h->dev_flag = (int*)dmalloc(sizeof(int));
    HZ_CU(cudaMemsetAsync(h->dev_flag, 0, sizeof(int), h->s2));
    const size_t n = n_dof(*p);
    h->c_pml = p->c_pml > 0 ? p->c_pml : mean_velocity(m_dev, n, h->s2);
    build_levels(h, m_dev);
    const size_t ps = prec_size(*p);
    const int R = p->max_rhs, m = p->gmres_m;
    Level& L = *h->sweep;
    const size_t nl = L.size();
    h->pr_r = dmalloc(ps * nl * R);
    h->pr_u = dmalloc(ps * nl * R);
    h->pr_u2 = dmalloc(ps * nl * R);
    h->pr_g = dmalloc(ps * nl * R);
    // transmission buffers [2][R][N_t]: the two layers passed between slabs
    h->pr_B1 = dmalloc(ps * 2 * R * L.nt());
    h->pr_B2 = dmalloc(ps * 2 * R * L.nt());
    HZ_CU(cudaMemsetAsync(h->pr_B1, 0, ps * 2 * R * L.nt(), h->s2));
    HZ_CU(cudaMemsetAsync(h->pr_B2, 0, ps * 2 * R * L.nt(), h->s2));
    if (p->sweep == HZ_SWEEP_NX) {
      const size_t nb = ps * 2 * R * L.nt() * (2 * (size_t)p->n_cell + 2);
      h->pr_Bnx = dmalloc(nb);
      HZ_CU(cudaMemsetAsync(h->pr_Bnx, 0, nb, h->s2));
    }
    if (p->two_grid) {
      h->tg_u = dmalloc(ps * n * R);
      h->tg_r = dmalloc(ps * n * R);
      h->tg_t = dmalloc(ps * n * R);
    }
    h->V = (c128*)dmalloc(sizeof(c128) * n * R * (m + 1));
    h->Z = (c128*)dmalloc(sizeof(c128) * n * R * m);
    h->W = (c128*)dmalloc(sizeof(c128) * n * R);
    h->R = (c128*)dmalloc(sizeof(c128) * n * R);
    h->red = (double*)dmalloc(sizeof(double) * gmres_red_doubles(m, R));
    h->hcol = (c128*)dmalloc(sizeof(c128) * 2 * R * (m + 2));
    HZ_CU(cudaStreamSynchronize(h->s2));
    h->stats.t_setup_s = now_s() - t0;
  });
  if (st != HZ_OK) {
    hz_destroy(h);
    return st;
  }
  *out = h;
  return HZ_OK;
}

hz_status hz_set_medium(hz_handle* h, const double* m_dev) {
  if (!h) return fail(nullptr, HZ_EINVAL, "handle is NULL");
  return guarded(h, [&] {
    if (!m_dev) throw Failure(HZ_EINVAL, "m_dev is NULL");
    // rebuild the level from scratch for the new medium (same grid)
    double t0 = now_s();
    const hz_params p = h->p;
    clear_graphs(h);
    free_level(h->fine);
    free_level(h->coarse);
    h->c_pml = p.c_pml > 0 ? p.c_pml : mean_velocity(m_dev, n_dof(p), h->s2);
    build_levels(h, m_dev);
    h->factored = false;
    h->stats.t_setup_s = now_s() - t0;
  });
}

hz_status hz_factor(hz_handle* h, void* stream) {
  if (!h) return fail(nullptr, HZ_EINVAL, "handle is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  return guarded(h, [&] {
    double t0 = now_s();
    h->factored = false;
    Level& L = *h->sweep;
    if (L.dim3d) {
      if (h->p.precision == HZ_MIXED)
        factor_level3d<float>(h, L, s);
      else
        factor_level3d<double>(h, L, s);
    } else {
      if (h->p.precision == HZ_MIXED)
        factor_level<float>(h, L, s);
      else
        factor_level<double>(h, L, s);
    }
    check_dev_flag(h, s);
    h->factored = true;
    h->stats.t_factor_s = now_s() - t0;
  });
}

hz_status hz_solve(hz_handle* h, const hz_c128* f_dev, hz_c128* u_dev, int n_rhs, void* stream,
                   hz_stats* stats) {
  if (!h) return fail(nullptr, HZ_EINVAL, "handle is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  hz_status st = guarded(h, [&] {
    if (!h->factored) throw Failure(HZ_ENOTFACTORED, "hz_solve before hz_factor");
    if (n_rhs < 1 || n_rhs > h->p.max_rhs) throw Failure(HZ_EINVAL, "n_rhs out of range");
    if (!f_dev || !u_dev) throw Failure(HZ_EINVAL, "NULL field pointer");
    double t0 = now_s();
    h->stats.precond_applies = 0;
    try {
      gmres_solve(h, (const c128*)f_dev, (c128*)u_dev, n_rhs, s);
    } catch (const Failure& f) {
      HZ_CU(cudaStreamSynchronize(s));
      h->stats.t_solve_s = now_s() - t0;
      h->stats.kernel_launches = h->launches;
      throw;
    }
    HZ_CU(cudaStreamSynchronize(s));
    h->stats.t_solve_s = now_s() - t0;
    h->stats.kernel_launches = h->launches;
  });
  if (stats) *stats = h->stats;
  return st;
}

hz_status hz_solve_host(hz_handle* h, const hz_c128* f_host, hz_c128* u_host, int n_rhs,
                        void* stream, hz_stats* stats) {
  if (!h) return fail(nullptr, HZ_EINVAL, "handle is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t n = h->fine.size() * n_rhs;
  hz_status st = guarded(h, [&] {
    if (n_rhs < 1 || n_rhs > h->p.max_rhs) throw Failure(HZ_EINVAL, "n_rhs out of range");
    if (!f_host || !u_host) throw Failure(HZ_EINVAL, "NULL field pointer");
    if (!h->stage_f) {   // allocated once, on the first host call
      const size_t cap = h->fine.size() * h->p.max_rhs;
      h->stage_f = (c128*)dmalloc(sizeof(c128) * cap);
      h->stage_u = (c128*)dmalloc(sizeof(c128) * cap);
    }
    HZ_CU(cudaMemcpyAsync(h->stage_f, f_host, sizeof(c128) * n, cudaMemcpyHostToDevice, s));
  });
  if (st == HZ_OK) {
    st = hz_solve(h, (const hz_c128*)h->stage_f, (hz_c128*)h->stage_u, n_rhs, stream, stats);
    if (st == HZ_OK || st == HZ_ENOTCONV) {
      hz_status st2 = guarded(h, [&] {
        HZ_CU(cudaMemcpyAsync(u_host, h->stage_u, sizeof(c128) * n, cudaMemcpyDeviceToHost, s));
        HZ_CU(cudaStreamSynchronize(s));
      });
      if (st2 != HZ_OK) st = st2;
    }
  }
  return st;
}

hz_status hz_apply(hz_handle* h, const hz_c128* u_dev, hz_c128* y_dev, int n_rhs, void* stream) {
  if (!h) return fail(nullptr, HZ_EINVAL, "handle is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  return guarded(h, [&] {
    if (n_rhs < 1 || n_rhs > h->p.max_rhs) throw Failure(HZ_EINVAL, "n_rhs out of range");
    if (!u_dev || !y_dev) throw Failure(HZ_EINVAL, "NULL field pointer");
    apply_fine64(h, (const c128*)u_dev, (c128*)y_dev, n_rhs, s);
    HZ_CU(cudaStreamSynchronize(s));
  });
}

hz_status hz_precond(hz_handle* h, const hz_c128* r_dev, hz_c128* z_dev, int n_rhs, void* stream) {
  if (!h) return fail(nullptr, HZ_EINVAL, "handle is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  return guarded(h, [&] {
    if (!h->factored) throw Failure(HZ_ENOTFACTORED, "hz_precond before hz_factor");
    if (n_rhs < 1 || n_rhs > h->p.max_rhs) throw Failure(HZ_EINVAL, "n_rhs out of range");
    if (!r_dev || !z_dev || r_dev == z_dev) throw Failure(HZ_EINVAL, "bad field pointers");
    precond_apply(h, (const c128*)r_dev, (c128*)z_dev, n_rhs, s);
    HZ_CU(cudaStreamSynchronize(s));
    check_dev_flag(h, s);
  });
}

hz_status hz_grad(hz_handle* h, const int* src_dev, int n_src, const int* rec_dev,
                         int n_rec, const hz_c128* d_dev, double* grad_dev, double* phi,
                         void* stream, hz_stats* stats) {
  if (!h) return fail(nullptr, HZ_EINVAL, "handle is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  hz_status st = guarded(h, [&] {
    if (!h->factored) throw Failure(HZ_ENOTFACTORED, "hz_grad before hz_factor");
    if (n_src < 1 || n_rec < 0) throw Failure(HZ_EINVAL, "need n_src >= 1 and n_rec >= 0");
    if (!src_dev || !grad_dev || !phi || (n_rec > 0 && (!rec_dev || !d_dev)))
      throw Failure(HZ_EINVAL, "NULL argument");
    double t0 = now_s();
    try {
      misfit_grad(h, src_dev, n_src, rec_dev, n_rec, (const c128*)d_dev, grad_dev, phi, s);
    } catch (const Failure& f) {
      cudaStreamSynchronize(s);
      h->stats.t_solve_s = now_s() - t0;
      h->stats.kernel_launches = h->launches;
      throw;
    }
    h->stats.t_solve_s = now_s() - t0;
    h->stats.kernel_launches = h->launches;
  });
  if (stats) *stats = h->stats;
  return st;
}

hz_status hz_slab_info(const hz_handle* h, int j, int* lo, int* hi, int* wl, int* wr, int* W) {
  if (!h || !h->sweep) return HZ_EINVAL;
  const Level& L = *h->sweep;
  if (j < 1 || j > L.J) return HZ_EINVAL;
  const Slab& S = L.slabs[j];
  if (lo) *lo = S.lo;
  if (hi) *hi = S.hi;
  if (wl) *wl = S.wl;
  if (wr) *wr = S.wr;
  if (W) *W = S.W;
  return HZ_OK;
}

hz_status hz_segment_layout(int ny, int segments, int max_auto, int* mid, int* P, int* S0,
                            int* NG, int* G0, int* seg_out, int seg_cap, int* grp_out,
                            int grp_cap) {
  if (!mid || !P || !S0 || !NG || !G0) return fail(nullptr, HZ_EINVAL, "NULL count pointer");
  if (ny < 3) return fail(nullptr, HZ_EINVAL, "a slab needs at least 3 rows");
  SegmentLayout L;
  try {
    L = segment_layout(ny, segments, max_auto);
  } catch (const Failure& f) {
    return fail(nullptr, f.st, f.msg);
  }
  *mid = L.mid;
  *P = L.P;
  *S0 = L.S0;
  *NG = L.NG;
  *G0 = L.G0;
  if ((seg_out && seg_cap < L.P) || (grp_out && grp_cap < L.NG))
    return fail(nullptr, HZ_EINVAL, "output capacity below the segment or group count");
  if (seg_out)
    for (int q = 0; q < L.P; ++q) {
      seg_out[4 * q] = L.seg[q].x;
      seg_out[4 * q + 1] = L.seg[q].y;
      seg_out[4 * q + 2] = L.seg[q].z;
      seg_out[4 * q + 3] = L.seg[q].w;
    }
  if (grp_out)
    for (int g = 0; g < L.NG; ++g) {
      grp_out[4 * g] = L.grp[g].x;
      grp_out[4 * g + 1] = L.grp[g].y;
      grp_out[4 * g + 2] = L.grp[g].z;
      grp_out[4 * g + 3] = L.grp[g].w;
    }
  return HZ_OK;
}

hz_status hz_slab_solve(hz_handle* h, int j, const hz_c128* f_dev, hz_c128* u_dev, int n_rhs,
                        void* stream) {
  if (!h) return fail(nullptr, HZ_EINVAL, "handle is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  void* tf = nullptr;
  void* tu = nullptr;
  hz_status st = guarded(h, [&] {
    if (!h->factored) throw Failure(HZ_ENOTFACTORED, "hz_slab_solve before hz_factor");
    Level& L = *h->sweep;
    if (j < 1 || j > L.J) throw Failure(HZ_EINVAL, "slab index out of range");
    if (n_rhs < 1 || n_rhs > h->p.max_rhs) throw Failure(HZ_EINVAL, "n_rhs out of range");
    if (!f_dev || !u_dev) throw Failure(HZ_EINVAL, "NULL field pointer");
    const size_t n = (size_t)n_rhs * L.nt() * L.slabs[j].W;
    if (h->p.precision == HZ_MIXED) {
      tf = dmalloc(sizeof(c64) * n);
      tu = dmalloc(sizeof(c64) * n);
      cast_copy<float, double>((const c128*)f_dev, (c64*)tf, n, s);
      if (L.dim3d)
        slab_solve_raw3d<float>(h, L, j, (const c64*)tf, (c64*)tu, n_rhs, s);
      else
        slab_solve_raw<float>(h, L, j, (const c64*)tf, (c64*)tu, n_rhs, s);
      cast_copy<double, float>((const c64*)tu, (c128*)u_dev, n, s);
    } else if (L.dim3d) {
      slab_solve_raw3d<double>(h, L, j, (const c128*)f_dev, (c128*)u_dev, n_rhs, s);
    } else {
      slab_solve_raw<double>(h, L, j, (const c128*)f_dev, (c128*)u_dev, n_rhs, s);
    }
    HZ_CU(cudaStreamSynchronize(s));
    check_dev_flag(h, s);
  });
  dfree(tf);
  dfree(tu);
  return st;
}

hz_status hz_get_stats(const hz_handle* h, hz_stats* out) {
  if (!h || !out) return HZ_EINVAL;
  *out = h->stats;
  out->kernel_launches = h->launches;
  return HZ_OK;
}

hz_status hz_enable_timing(hz_handle* h, int on) {
  if (!h) return HZ_EINVAL;
  return guarded(h, [&] {
    for (auto& kv : h->timing.tags) {
      TagTiming& t = kv.second;
      for (size_t i = 0; i < t.used; ++i) HZ_CU(cudaEventSynchronize(t.ev[i].second));
      t.used = 0;
      t.ms = 0;
      t.launches = 0;
      t.bytes = 0;
    }
    h->timing.on = on != 0;
  });
}

hz_status hz_kernel_timing(hz_handle* h, const char* tag, double* ms, long long* launches,
                           double* bytes) {
  if (!h || !tag) return HZ_EINVAL;
  return guarded(h, [&] {
    auto it = h->timing.tags.find(tag);
    double m = 0, b = 0;
    long long n = 0;
    if (it != h->timing.tags.end()) {
      TagTiming& t = it->second;
      double acc = 0;
      for (size_t i = 0; i < t.used; ++i) {
        HZ_CU(cudaEventSynchronize(t.ev[i].second));
        float x = 0;
        HZ_CU(cudaEventElapsedTime(&x, t.ev[i].first, t.ev[i].second));
        acc += x;
      }
      t.ms += acc;
      t.used = 0;
      m = t.ms; n = t.launches; b = t.bytes;
    }
    if (ms) *ms = m;
    if (launches) *launches = n;
    if (bytes) *bytes = b;
  });
}

void hz_destroy(hz_handle* h) {
  if (!h) return;
  cudaDeviceSynchronize();
  clear_graphs(h);
  free_level(h->fine);
  free_level(h->coarse);
  release_work(h);
  dfree(h->dev_flag);
  if (h->s2) cudaStreamDestroy(h->s2);
  if (h->evA) cudaEventDestroy(h->evA);
  if (h->evB) cudaEventDestroy(h->evB);
  for (auto& kv : h->timing.tags)
    for (auto& e : kv.second.ev) {
      cudaEventDestroy(e.first);
      cudaEventDestroy(e.second);
    }
  dfree(h->stage_f);
  dfree(h->stage_u);
  dfree(h->gr_b);
  dfree(h->gr_u);
  dfree(h->gr_mu);
  dfree(h->gr_phi);
  dfree(h->gm_state);
  cudaGetLastError();
  delete h;
}

}  // extern "C"
