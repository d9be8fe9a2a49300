// Entry points of libhpt that enqueue device work: hpt_eval, hpt_paths_init,
// hpt_step, hpt_track, hpt_polish, hpt_adjoint, hpt_euler_newton.
#include <string.h>

#include <algorithm>

#include "hpt_internal.h"

namespace hpt {

hpt_paths offset_paths(const hpt_paths& S, int64_t q0, int n, size_t cs) {
  hpt_paths o = S;
  o.y = (char*)S.y + q0 * n * cs;
  o.y_acc = (char*)S.y_acc + q0 * n * cs;
  o.dE_acc = (char*)S.dE_acc + q0 * n * cs;
  o.tau = S.tau + q0;
  o.dtau = S.dtau + q0;
  o.tau_acc = S.tau_acc + q0;
  o.status = S.status + q0;
  o.steps = S.steps + q0;
  o.accepts = S.accepts + q0;
  o.rejects = S.rejects + q0;
  o.streak = S.streak + q0;
  if (S.y_prev) o.y_prev = (char*)S.y_prev + q0 * n * cs;
  if (S.dE_prev) o.dE_prev = (char*)S.dE_prev + q0 * n * cs;
  if (S.tau_prev) o.tau_prev = S.tau_prev + q0;
  if (S.hermite) o.hermite = S.hermite + q0;
  return o;
}

namespace {

inline size_t csize(const hpt_system s) { return s->prec == HPT_FP64 ? 16 : 8; }

cudaError_t eval_form(hpt_system s, int64_t p, const void* y, const double* tau, int tau_is_t,
                      const EvalOut& out, cudaStream_t st) {
  return s->prec == HPT_FP64 ? launch_eval_fp64(s, p, y, tau, tau_is_t, out, st)
                             : launch_eval_mixed(s, p, y, tau, tau_is_t, out, st);
}

hpt_status step_impl(hpt_system s, int64_t p, const hpt_paths& S, int32_t nsteps,
                     const hpt_params& prm, cudaStream_t st) {
  const int n = s->n, nv = s->nv;
  const int64_t chunk = std::min<int64_t>(p, kChunk);
  // scratch: extended Jacobian of a chunk, then the FP64 re-solve list
  const size_t ext_bytes = (ext_entries(chunk, nv) * csize(s) + 255) / 256 * 256;
  hpt_status rc = ensure_scratch(s, ext_bytes + 256 + (size_t)chunk * sizeof(int64_t));
  if (rc) return rc;
  int32_t* redo_count = (int32_t*)((char*)s->d_scratch + ext_bytes);
  int64_t* redo_list = (int64_t*)((char*)s->d_scratch + ext_bytes + 256);
  for (int r = 0; r < nsteps; ++r) {
    for (int64_t q0 = 0; q0 < p; q0 += chunk) {
      const int64_t cnt = std::min(chunk, p - q0);
      hpt_paths sub = offset_paths(S, q0, nv, csize(s));
      EvalOut out;
      out.ext = s->d_scratch;
      cudaError_t e = eval_form(s, cnt, sub.y, sub.tau, 0, out, st);
      if (e != cudaSuccess) return cuda_fail(e, "evaluation launch");
      if (s->proj) {   // Algorithm 3 by QR, projective step control
        e = launch_qr_step(s, cnt, s->d_scratch, sub, prm, st);
        if (e != cudaSuccess) return cuda_fail(e, "QR step launch");
        continue;
      }
      StepArgs a;
      a.n = n;
      a.p = cnt;
      a.ext = s->d_scratch;
      a.st = sub;
      a.prm = prm;
      a.err = s->d_err;
      a.redo_count = redo_count;
      a.redo_list = redo_list;
      e = launch_solve_update(s, a, st);
      if (e != cudaSuccess) return cuda_fail(e, "solve launch");
    }
  }
  return HPT_OK;
}

// The polish runs on the affine system (a projective handle keeps its FP64
// constants in s->affine) with the scratch of s.
hpt_status polish_impl(hpt_system s, int64_t p, void* x, int32_t* done, float* last, const hpt_params& prm,
                       cudaStream_t st) {
  const hpt_system a = s->affine ? s->affine : s;
  const int64_t chunk = std::min<int64_t>(p, kChunk);
  hpt_status rc = ensure_scratch(s, ext_entries(chunk, a->n) * 16);
  if (rc) return rc;
  return polish_paths(a, p, x, done, last, prm, s->d_scratch, chunk, st);
}

}  // namespace

hpt_status polish_paths(hpt_system s, int64_t p, void* x, int32_t* done, float* last, const hpt_params& prm,
                        void* ext, int64_t chunk, cudaStream_t st) {
  const int n = s->n;
  cudaError_t e0 = cudaMemsetAsync(last, 0, (size_t)p * sizeof(float), st);
  if (e0 != cudaSuccess) return cuda_fail(e0, "polish init");
  for (int it = 0; it < prm.polish_iters; ++it) {
    for (int64_t q0 = 0; q0 < p; q0 += chunk) {
      const int64_t cnt = std::min(chunk, p - q0);
      EvalOut out;
      out.ext = ext;
      void* xq = (char*)x + q0 * n * 16;
      cudaError_t e = launch_eval_fp64(s, cnt, xq, nullptr, 0, out, st);
      if (e != cudaSuccess) return cuda_fail(e, "polish evaluation launch");
      e = launch_newton_update(s, cnt, ext, xq, done + q0, last + q0, prm.polish_tol, st);
      if (e != cudaSuccess) return cuda_fail(e, "polish update launch");
    }
  }
  return HPT_OK;
}

hpt_status check_params(const hpt_params* prm) {
  if (!prm) { set_error("params is NULL"); return HPT_EINVAL; }
  if (!(prm->tol_accept > 0) || !(prm->dtau_init > 0) || !(prm->dtau_min > 0) ||
      !(prm->dtau_max >= prm->dtau_min) || !(prm->grow >= 1) || !(prm->shrink > 0 && prm->shrink < 1) ||
      prm->grow_after < 1 || prm->max_steps < 1 || !(prm->div_bound > 1) || !(prm->polish_tol > 0) ||
      prm->polish_iters < 0 || (prm->predictor != 0 && prm->predictor != 1)) {
    set_error("params out of range");
    return HPT_EINVAL;
  }
  return HPT_OK;
}

hpt_status check_state(const hpt_paths* S, const hpt_params* prm) {
  if (!S->y || !S->y_acc || !S->dE_acc || !S->tau || !S->dtau || !S->tau_acc || !S->status ||
      !S->steps || !S->accepts || !S->rejects || !S->streak) {
    set_error("NULL pointer in the path state");
    return HPT_EINVAL;
  }
  if (prm->predictor == 1 && (!S->y_prev || !S->dE_prev || !S->tau_prev || !S->hermite)) {
    set_error("the Hermite predictor needs y_prev, dE_prev, tau_prev and hermite in the path state");
    return HPT_EINVAL;
  }
  return HPT_OK;
}

hpt_status cuda_fail(cudaError_t e, const char* what) {
  set_error("%s: %s", what, cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? HPT_ENOMEM : HPT_ECUDA;
}

namespace {

hpt_status check_sys(hpt_system s) {
  if (!s) { set_error("NULL handle"); return HPT_EINVAL; }
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != s->device) {
    set_error("the handle belongs to device %d, current device is %d", s->device, dev);
    return HPT_EINVAL;
  }
  return HPT_OK;
}

}  // namespace
}  // namespace hpt

using namespace hpt;

extern "C" {

hpt_status hpt_eval(hpt_system s, int64_t p, const void* y, const double* t, void* H, void* Hy,
                    void* Ht, void* stream) {
  hpt_status rc = check_sys(s);
  if (rc) return rc;
  if (p < 0) { set_error("p < 0"); return HPT_EINVAL; }
  if (p == 0) return HPT_OK;
  if (!y || !t) { set_error("y or t is NULL"); return HPT_EINVAL; }
  if (!H && !Hy && !Ht) return HPT_OK;
  EvalOut out;
  out.H = H;
  out.Hy = Hy;
  out.Ht = Ht;
  cudaError_t e = eval_form(s, p, y, t, 1, out, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "evaluation launch");
  return HPT_OK;
}

hpt_status hpt_paths_init(hpt_system s, int64_t p, const void* y0, const hpt_params* prm,
                          const hpt_paths* S, void* stream) {
  hpt_status rc = check_sys(s);
  if (rc) return rc;
  if ((rc = check_params(prm))) return rc;
  if (p < 0 || !S) { set_error("bad p or state"); return HPT_EINVAL; }
  if (p == 0) return HPT_OK;
  if (!y0) { set_error("y0 is NULL"); return HPT_EINVAL; }
  if ((rc = check_state(S, prm))) return rc;
  double tau0 = 0;
  hpt_get_info(s, nullptr, nullptr, nullptr, prm->eps0, &tau0);
  cudaError_t e = s->proj ? launch_paths_init_proj(s, p, y0, tau0, *prm, *S, (cudaStream_t)stream)
                          : launch_paths_init(s, p, y0, tau0, *prm, *S, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "init launch");
  return HPT_OK;
}

hpt_status hpt_step(hpt_system s, int64_t p, const hpt_paths* S, int32_t nsteps,
                    const hpt_params* prm, void* stream) {
  hpt_status rc = check_sys(s);
  if (rc) return rc;
  if ((rc = check_params(prm))) return rc;
  if (p < 0 || !S || nsteps < 0) { set_error("bad p, state or nsteps"); return HPT_EINVAL; }
  if (p == 0 || nsteps == 0) return HPT_OK;
  if ((rc = check_state(S, prm))) return rc;
  return step_impl(s, p, *S, nsteps, *prm, (cudaStream_t)stream);
}

hpt_status hpt_track(hpt_system s, int64_t p, const void* y0, const hpt_params* prm, void* x_out,
                     int32_t* status_out, int32_t* steps_out, void* stream) {
  hpt_status rc = check_sys(s);
  if (rc) return rc;
  if ((rc = check_params(prm))) return rc;
  if (p < 0) { set_error("p < 0"); return HPT_EINVAL; }
  if (p == 0) return HPT_OK;
  if (!y0 || !x_out) { set_error("y0 or x_out is NULL"); return HPT_EINVAL; }
  if (s->prec == HPT_MIXED && !s->proj) {
    // the mixed form tracks through a one-system batch (cached in the handle):
    // finished paths leave the launches after every round instead of being
    // evaluated until the last path ends; per path the arithmetic is the same
    if (!s->self_batch) {
      hpt_batch b = nullptr;
      if ((rc = hpt_batch_create(1, &s, &b))) return rc;
      s->self_batch = b;
    }
    return hpt_batch_track(s->self_batch, &p, y0, prm, x_out, status_out, steps_out, stream);
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int n = s->nv;   // state entries per path (homogeneous coordinates in the projective form)
  const size_t cs = csize(s);
  // state layout inside the library's track scratch
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off += (bytes + 255) / 256 * 256;
    return o;
  };
  const size_t o_y = take(p * n * cs), o_ya = take(p * n * cs), o_de = take(p * n * cs);
  const size_t o_yp = take(p * n * cs), o_dp = take(p * n * cs), o_tp = take(p * 8), o_hf = take(p * 4);
  const size_t o_tau = take(p * 8), o_dt = take(p * 8), o_ta = take(p * 8);
  const size_t o_st = take(p * 4), o_sp = take(p * 4), o_ac = take(p * 4), o_rj = take(p * 4),
               o_sk = take(p * 4), o_done = take(p * 4), o_last = take(p * 4), o_cnt = take(4);
  if ((rc = ensure_track(s, off))) return rc;
  char* b = (char*)s->d_track;
  hpt_paths S;
  S.y = b + o_y;
  S.y_acc = b + o_ya;
  S.dE_acc = b + o_de;
  S.tau = (double*)(b + o_tau);
  S.dtau = (double*)(b + o_dt);
  S.tau_acc = (double*)(b + o_ta);
  S.status = (int32_t*)(b + o_st);
  S.steps = (int32_t*)(b + o_sp);
  S.accepts = (int32_t*)(b + o_ac);
  S.rejects = (int32_t*)(b + o_rj);
  S.streak = (int32_t*)(b + o_sk);
  S.y_prev = b + o_yp;
  S.dE_prev = b + o_dp;
  S.tau_prev = (double*)(b + o_tp);
  S.hermite = (int32_t*)(b + o_hf);
  int32_t* done = (int32_t*)(b + o_done);
  float* last = (float*)(b + o_last);
  int32_t* cnt = (int32_t*)(b + o_cnt);
  if ((rc = hpt_paths_init(s, p, y0, prm, &S, stream))) return rc;
  const int every = prm->check_every > 0 ? prm->check_every : 32;
  int64_t total = 0;
  for (;;) {
    if ((rc = step_impl(s, p, S, every, *prm, st))) return rc;
    total += every;
    cudaError_t e = launch_count_active(p, S.status, cnt, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->h_count, cnt, 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "active-path count");
    if (*s->h_count == 0 || total > (int64_t)prm->max_steps + every) break;
  }
  cudaError_t e = s->proj ? launch_finish_track_proj(s, p, S, x_out, status_out, steps_out, done, st)
                          : launch_finish_track(s, p, S, x_out, status_out, steps_out, done, st);
  if (e != cudaSuccess) return cuda_fail(e, "track output");
  if ((rc = polish_impl(s, p, x_out, done, last, *prm, st))) return rc;
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "track");
  return HPT_OK;
}

hpt_status hpt_polish(hpt_system s, int64_t p, void* x, const int32_t* status, const hpt_params* prm,
                      void* stream) {
  hpt_status rc = check_sys(s);
  if (rc) return rc;
  if ((rc = check_params(prm))) return rc;
  if (p < 0) { set_error("p < 0"); return HPT_EINVAL; }
  if (p == 0) return HPT_OK;
  if (!x) { set_error("x is NULL"); return HPT_EINVAL; }
  const size_t done_bytes = ((size_t)p * 4 + 255) / 256 * 256;
  if ((rc = ensure_track(s, done_bytes + (size_t)p * 4))) return rc;
  int32_t* done = (int32_t*)s->d_track;
  cudaError_t e = launch_init_done(p, status, done, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "polish init");
  return polish_impl(s, p, x, done, (float*)((char*)s->d_track + done_bytes), *prm, (cudaStream_t)stream);
}

hpt_status hpt_adjoint(hpt_system s, int64_t p, const void* x, const void* gx, void* gc, void* stream) {
  hpt_status rc = check_sys(s);
  if (rc) return rc;
  if (p < 0 || !gc) { set_error("bad p or gc is NULL"); return HPT_EINVAL; }
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaMemsetAsync(gc, 0, (size_t)s->M * 16, st);
  if (e != cudaSuccess) return cuda_fail(e, "adjoint init");
  if (p == 0) return HPT_OK;
  if (!x || !gx) { set_error("x or gx is NULL"); return HPT_EINVAL; }
  const hpt_system a = s->affine ? s->affine : s;   // solutions are affine points
  const int n = a->n;
  const int64_t chunk = std::min<int64_t>(p, 8192);
  const size_t ext_bytes = (ext_entries(chunk, n) * 16 + 255) / 256 * 256;
  const size_t contrib_bytes = ((size_t)chunk * s->M * 16 + 255) / 256 * 256;
  if ((rc = ensure_scratch(s, ext_bytes + contrib_bytes + adjoint_part_bytes(s->M)))) return rc;
  void* contrib = (char*)s->d_scratch + ext_bytes;
  void* part = (char*)contrib + contrib_bytes;
  for (int64_t q0 = 0; q0 < p; q0 += chunk) {
    const int64_t cnt = std::min(chunk, p - q0);
    EvalOut out;
    out.ext = s->d_scratch;
    const void* xq = (const char*)x + q0 * n * 16;
    e = launch_eval_fp64(a, cnt, xq, nullptr, 0, out, st);
    if (e != cudaSuccess) return cuda_fail(e, "adjoint evaluation launch");
    e = launch_adjoint(a, cnt, s->d_scratch, xq, (const char*)gx + q0 * n * 16, contrib, part, gc, st);
    if (e != cudaSuccess) return cuda_fail(e, "adjoint launch");
  }
  return HPT_OK;
}

hpt_status hpt_check_bounded_wait(hpt_system s, void* stream) {
  hpt_status rc = check_sys(s);
  if (rc) return rc;
  cudaError_t e = launch_bounded_wait_probe(s->d_err, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "bounded-wait probe launch");
  return HPT_OK;
}

hpt_status hpt_euler_newton(hpt_system s, int64_t p, const void* y, const double* tau, void* dE, void* dN,
                            int32_t* ok, void* stream) {
  hpt_status rc = check_sys(s);
  if (rc) return rc;
  if (p < 0) { set_error("p < 0"); return HPT_EINVAL; }
  if (p == 0) return HPT_OK;
  if (!y || !tau || !dE || !dN || !ok) { set_error("NULL pointer argument"); return HPT_EINVAL; }
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t chunk = std::min<int64_t>(p, kChunk);
  if ((rc = ensure_scratch(s, ext_entries(chunk, s->nv) * csize(s)))) return rc;
  const size_t cs = csize(s);
  for (int64_t q0 = 0; q0 < p; q0 += chunk) {
    const int64_t cnt = std::min(chunk, p - q0);
    const size_t vo = (size_t)q0 * s->nv * cs;
    EvalOut out;
    out.ext = s->d_scratch;
    cudaError_t e = eval_form(s, cnt, (const char*)y + vo, tau + q0, 0, out, st);
    if (e != cudaSuccess) return cuda_fail(e, "evaluation launch");
    e = launch_qr_directions(s, cnt, s->d_scratch, (const char*)y + vo, (char*)dE + vo, (char*)dN + vo, ok + q0, st);
    if (e != cudaSuccess) return cuda_fail(e, "QR launch");
  }
  return HPT_OK;
}

}  // extern "C"
