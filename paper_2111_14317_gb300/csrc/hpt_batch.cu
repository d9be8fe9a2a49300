// Batching form: the paths of many mixed-form systems (n may differ) tracked
// together.  Parallelism across systems on top of the point-level batching of
// Section 5 (problem (d) of Section 1).
//
// Layout.  Paths are numbered system by system (system s owns paths
// pb[s] .. pb[s]+paths[s]-1); their variables are concatenated (vofs[path] =
// offset of the first one).  A position list names the live paths, padded per
// system to whole 128-position tiles (entry -1 = padding), so every tile
// belongs to one system (tile_sys).  Systems are ordered by lane-group shape
// bucket (n <= 8, <= 16, <= 24, <= 32), inside a bucket by decreasing evaluation
// cost, so each solve launch covers one contiguous position range and the
// evaluation kernel's round-robin tile walk meets the large tiles first.
//
// A round is K x (evaluation over every position; per bucket the FP32 solve
// over its range; the FP64 re-solve list) followed by the compaction (count,
// scan, scatter) and a read-back of the position count.  It is captured once
// into a CUDA graph on the batch's own stream and replayed until the count
// is 0 or the step budget is spent.
#include <string.h>

#include <algorithm>
#include <chrono>
#include <numeric>
#include <vector>

#include "hpt_internal.h"

namespace hpt {
constexpr int kBuckets = 4;   // n <= 8, <= 16, <= 24, <= 32
inline int bucket_of(int n) { return n <= 8 ? 0 : (n <= 16 ? 1 : (n <= 24 ? 2 : 3)); }
// Order indices of the first and last system of each shape bucket (-1: the
// bucket is empty); order is sorted by bucket, so a bucket's tiles are one
// contiguous range.
struct BucketSpan {
  int first[kBuckets], last[kBuckets];
};
}  // namespace hpt

struct hpt_batch_s {
  int device = 0;
  int nsys = 0;
  std::vector<hpt_system> sys;
  std::vector<int> sys_n;
  std::vector<int> bucket;        // lane-group shape of each system
  std::vector<int32_t> order;     // systems in position order
  hpt::BucketSpan span{};
  hpt::MixedSys maxs{};   // the largest of each operand dimension
  int tmem_cols = 0;
  int nmax = 0;
  int redo_shape = 0;

  // constants on the device
  uint8_t* d_chunks = nullptr;
  hpt::MixedSys* d_tab = nullptr;
  hpt::Fp64Sys* d_f64 = nullptr;
  int32_t* d_sys_n = nullptr;
  int32_t* d_order = nullptr;
  int32_t* d_err = nullptr;

  // per-problem state (grown on demand)
  void* d_state = nullptr;
  size_t state_bytes = 0;
  int32_t* h_ctl = nullptr;       // pinned copy of the control words

  cudaStream_t own = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;

  // captured round and the key it was captured for
  cudaGraphExec_t exec = nullptr;
  void* key_state = nullptr;
  std::vector<int64_t> key_paths;
  hpt_batch_tuning key_tune{0, 0, 0};
  hpt_params key_prm{};

  hpt_batch_tuning tune{16, 2, 8};
  int64_t rounds = 0, position_steps = 0;
  int32_t kernels_per_round = 0;
};

namespace hpt {
namespace {

// control words: [0] positions, [1 + b] bucket b's first position, [1 + kBuckets + b] its end
constexpr int kCtlWords = 2 + 2 * kBuckets;

// One block per system: the system's live paths (flag == want) in order,
// into tmp at the system's own path range; cnt[s] = their number.
__global__ void compact_count_kernel(const int64_t* __restrict__ pb, const int32_t* __restrict__ np,
                                     const int32_t* __restrict__ flag, int32_t want, int64_t* __restrict__ tmp,
                                     int32_t* __restrict__ cnt) {
  __shared__ int wsum[8];
  const int s = blockIdx.x;
  const int64_t base = pb[s];
  const int p = np[s];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int total = 0;
  for (int i0 = 0; i0 < p; i0 += 256) {
    const int i = i0 + threadIdx.x;
    const bool live = i < p && flag[base + i] == want;
    const unsigned bal = __ballot_sync(0xffffffffu, live);
    if (lane == 0) wsum[warp] = __popc(bal);
    __syncthreads();
    int before = total;
    for (int w = 0; w < warp; ++w) before += wsum[w];
    int chunk = 0;
    for (int w = 0; w < 8; ++w) chunk += wsum[w];
    if (live) tmp[base + before + __popc(bal & ((1u << lane) - 1u))] = base + i;
    total += chunk;
    __syncthreads();
  }
  if (threadIdx.x == 0) cnt[s] = total;
}

// One block: tiles per system in position order -> tile_base, the bucket
// ranges and the position count (ctl).
__global__ void compact_scan_kernel(int nsys, const int32_t* __restrict__ order, BucketSpan bs,
                                    const int32_t* __restrict__ cnt, int32_t* __restrict__ tile_base,
                                    int32_t* __restrict__ ctl) {
  __shared__ int part[1024];
  const int t = threadIdx.x;
  const int per = (nsys + 1023) / 1024;
  const int lo = min(nsys, t * per), hi = min(nsys, lo + per);
  int sum = 0;
  for (int i = lo; i < hi; ++i) sum += (cnt[order[i]] + 127) / 128;
  part[t] = sum;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {   // inclusive scan
    const int v = t >= o ? part[t - o] : 0;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  int run = part[t] - sum;
  for (int i = lo; i < hi; ++i) {
    const int s = order[i];
    tile_base[s] = run;
    run += (cnt[s] + 127) / 128;
  }
  __syncthreads();
  if (t < kBuckets) {
    int begin = 0, end = 0;
    if (bs.first[t] >= 0) {
      const int sf = order[bs.first[t]], sl = order[bs.last[t]];
      begin = tile_base[sf];
      end = tile_base[sl] + (cnt[sl] + 127) / 128;
    }
    ctl[1 + t] = begin * 128;
    ctl[1 + kBuckets + t] = end * 128;
  }
  if (t == 0) ctl[0] = part[1023] * 128;
}

// One block per system: its live paths and padding into the list, its tiles
// into tile_sys.
__global__ void compact_scatter_kernel(const int64_t* __restrict__ pb, const int64_t* __restrict__ tmp,
                                       const int32_t* __restrict__ cnt, const int32_t* __restrict__ tile_base,
                                       int64_t* __restrict__ list, int32_t* __restrict__ tile_sys) {
  const int s = blockIdx.x;
  const int c = cnt[s];
  const int ntile = (c + 127) / 128;
  const int64_t q0 = (int64_t)tile_base[s] * 128;
  for (int i = threadIdx.x; i < ntile * 128; i += blockDim.x) list[q0 + i] = i < c ? tmp[pb[s] + i] : -1;
  for (int i = threadIdx.x; i < ntile; i += blockDim.x) tile_sys[tile_base[s] + i] = s;
}

__global__ void fill_vofs_kernel(int64_t p, int n, int64_t vb, int64_t* __restrict__ vofs) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < p) vofs[i] = vb + i * n;
}

// Problem geometry and the state carve-up of one call.
struct Problem {
  std::vector<int64_t> pb, vb;   // path and variable offsets per system
  int64_t P = 0, V = 0;          // paths, variables
  int64_t cap = 0;               // list capacity (positions)
  int64_t cap_bucket[kBuckets] = {0, 0, 0, 0};
  int64_t pmax = 0;              // largest paths[s]
  // byte offsets in d_state
  size_t o_y, o_ya, o_de, o_yp, o_dp, o_tp, o_hf, o_tau, o_dt, o_ta, o_st, o_sp, o_ac, o_rj, o_sk, o_done, o_last, o_vofs,
      o_pb, o_np, o_tmp, o_cnt, o_tb, o_list, o_tsys, o_ctl, o_rc, o_rl, o_ext, total;
};

Problem plan(const hpt_batch_s* b, const int64_t* paths) {
  Problem q;
  q.pb.resize(b->nsys);
  q.vb.resize(b->nsys);
  for (int s = 0; s < b->nsys; ++s) {
    q.pb[s] = q.P;
    q.vb[s] = q.V;
    q.P += paths[s];
    q.V += paths[s] * b->sys_n[s];
    const int64_t tiles = (paths[s] + 127) / 128;
    q.cap += tiles * 128;
    q.cap_bucket[b->bucket[s]] += tiles * 128;
    q.pmax = std::max(q.pmax, paths[s]);
  }
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off += (bytes + 255) / 256 * 256;
    return o;
  };
  const size_t P = (size_t)std::max<int64_t>(q.P, 1), V = (size_t)std::max<int64_t>(q.V, 1);
  q.o_y = take(V * 8);
  q.o_ya = take(V * 8);
  q.o_de = take(V * 8);
  q.o_yp = take(V * 8);   // the accepted point before the last one (Hermite predictor)
  q.o_dp = take(V * 8);
  q.o_tp = take(P * 8);
  q.o_hf = take(P * 4);
  q.o_tau = take(P * 8);
  q.o_dt = take(P * 8);
  q.o_ta = take(P * 8);
  q.o_st = take(P * 4);
  q.o_sp = take(P * 4);
  q.o_ac = take(P * 4);
  q.o_rj = take(P * 4);
  q.o_sk = take(P * 4);
  q.o_done = take(P * 4);
  q.o_last = take(P * 4);
  q.o_vofs = take(P * 8);
  q.o_pb = take((size_t)b->nsys * 8);
  q.o_np = take((size_t)b->nsys * 4);
  q.o_tmp = take(P * 8);
  q.o_cnt = take((size_t)b->nsys * 4);
  q.o_tb = take((size_t)b->nsys * 4);
  q.o_list = take((size_t)std::max<int64_t>(q.cap, 128) * 8);
  q.o_tsys = take((size_t)std::max<int64_t>(q.cap / 128, 1) * 4);
  q.o_ctl = take(kCtlWords * 4);
  q.o_rc = take(4);
  q.o_rl = take((size_t)std::max<int64_t>(q.cap, 1) * 8);
  // extended Jacobian of every position: complex64 while tracking,
  // complex128 while polishing
  q.o_ext = take(ext_entries(std::max<int64_t>(q.cap, 1), b->nmax) * 16);
  q.total = off;
  return q;
}

hpt_paths state_of(const hpt_batch_s* b, const Problem& q) {
  char* d = (char*)b->d_state;
  hpt_paths S;
  S.y = d + q.o_y;
  S.y_acc = d + q.o_ya;
  S.dE_acc = d + q.o_de;
  S.tau = (double*)(d + q.o_tau);
  S.dtau = (double*)(d + q.o_dt);
  S.tau_acc = (double*)(d + q.o_ta);
  S.status = (int32_t*)(d + q.o_st);
  S.steps = (int32_t*)(d + q.o_sp);
  S.accepts = (int32_t*)(d + q.o_ac);
  S.rejects = (int32_t*)(d + q.o_rj);
  S.streak = (int32_t*)(d + q.o_sk);
  S.y_prev = d + q.o_yp;
  S.dE_prev = d + q.o_dp;
  S.tau_prev = (double*)(d + q.o_tp);
  S.hermite = (int32_t*)(d + q.o_hf);
  return S;
}

// The state of system s alone (its paths start at pb, variables at vb).
hpt_paths sub_state(const hpt_paths& S, int64_t pb, int64_t vb) {
  hpt_paths o = S;
  o.y = (char*)S.y + vb * 8;
  o.y_acc = (char*)S.y_acc + vb * 8;
  o.dE_acc = (char*)S.dE_acc + vb * 8;
  o.tau = S.tau + pb;
  o.dtau = S.dtau + pb;
  o.tau_acc = S.tau_acc + pb;
  o.status = S.status + pb;
  o.steps = S.steps + pb;
  o.accepts = S.accepts + pb;
  o.rejects = S.rejects + pb;
  o.streak = S.streak + pb;
  o.y_prev = (char*)S.y_prev + vb * 8;
  o.dE_prev = (char*)S.dE_prev + vb * 8;
  o.tau_prev = S.tau_prev + pb;
  o.hermite = S.hermite + pb;
  return o;
}

// The compaction kernels (3 launches) on stream st: the paths whose flag
// (status while tracking, done while polishing) equals want.
cudaError_t enqueue_compaction(const hpt_batch_s* b, const Problem& q, const int32_t* flag, int32_t want,
                               cudaStream_t st) {
  char* d = (char*)b->d_state;
  compact_count_kernel<<<b->nsys, 256, 0, st>>>((const int64_t*)(d + q.o_pb), (const int32_t*)(d + q.o_np), flag,
                                                want, (int64_t*)(d + q.o_tmp), (int32_t*)(d + q.o_cnt));
  compact_scan_kernel<<<1, 1024, 0, st>>>(b->nsys, b->d_order, b->span, (const int32_t*)(d + q.o_cnt),
                                          (int32_t*)(d + q.o_tb), (int32_t*)(d + q.o_ctl));
  compact_scatter_kernel<<<b->nsys, 256, 0, st>>>((const int64_t*)(d + q.o_pb), (const int64_t*)(d + q.o_tmp),
                                                  (const int32_t*)(d + q.o_cnt), (const int32_t*)(d + q.o_tb),
                                                  (int64_t*)(d + q.o_list), (int32_t*)(d + q.o_tsys));
  return cudaGetLastError();
}

// FP32 solve shape of bucket bk: 8-lane groups with 1, 2 or 3 rows per lane
// (n <= 8, 16, 24) or 32-lane groups; the n <= 24 bucket takes 32-lane
// groups instead when the tuning says so.
int fp32_shape(const hpt_batch_s* b, int bk) {
  if (bk < 2) return bk;
  if (bk == 2) return b->tune.solve_lanes_n17_24 == 8 ? kShape8x3 : 2;
  return 2;
}

// K steps and the compaction on st (captured by the caller).
cudaError_t enqueue_round(hpt_batch_s* b, const Problem& q, const hpt_params& prm, cudaStream_t st,
                          int32_t* kernels) {
  char* d = (char*)b->d_state;
  const hpt_paths S = state_of(b, q);
  int32_t* ctl = (int32_t*)(d + q.o_ctl);
  PathMap pm;
  pm.list = (const int64_t*)(d + q.o_list);
  pm.tile_sys = (const int32_t*)(d + q.o_tsys);
  pm.sys_n = b->d_sys_n;
  pm.vofs = (const int64_t*)(d + q.o_vofs);
  pm.npos = ctl;
  pm.nmax = b->nmax;
  pm.sys_tab = b->d_tab;
  int32_t nk = 0;
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < b->tune.steps_per_round && e == cudaSuccess; ++k) {
    e = cudaMemsetAsync(d + q.o_rc, 0, 4, st);
    if (e != cudaSuccess) break;
    e = launch_eval_mixed_map(nullptr, b->maxs, b->tmem_cols, b->d_chunks, q.cap, S.y, S.tau, pm, d + q.o_ext,
                              b->d_err, b->tune.eval_ctas_per_sm, st);
    ++nk;
    StepArgs a;
    a.n = b->nmax;
    a.ext = d + q.o_ext;
    a.st = S;
    a.prm = prm;
    a.err = b->d_err;
    a.redo_count = (int32_t*)(d + q.o_rc);
    a.redo_list = (int64_t*)(d + q.o_rl);
    for (int bk = 0; bk < kBuckets && e == cudaSuccess; ++bk) {
      if (!q.cap_bucket[bk]) continue;
      a.p = q.cap_bucket[bk];
      a.map = pm;
      a.map.pos_begin = ctl + 1 + bk;
      a.map.npos = ctl + 1 + kBuckets + bk;
      e = launch_solve_fp32_shape(fp32_shape(b, bk), a, st);
      ++nk;
    }
    if (e != cudaSuccess) break;
    a.p = q.cap;
    a.map = pm;
    e = launch_redo_fp64_shape(b->redo_shape, a, st);
    ++nk;
  }
  if (e == cudaSuccess) e = enqueue_compaction(b, q, S.status, HPT_PATH_ACTIVE, st);
  nk += 3;
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->h_ctl, ctl, kCtlWords * 4, cudaMemcpyDeviceToHost, st);
  *kernels = nk;
  return e;
}

bool same_prm(const hpt_params& a, const hpt_params& b) { return memcmp(&a, &b, sizeof(hpt_params)) == 0; }

hpt_status ensure_state(hpt_batch_s* b, size_t bytes) {
  if (bytes <= b->state_bytes) return HPT_OK;
  if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
  cudaFree(b->d_state);
  b->d_state = nullptr;
  b->state_bytes = 0;
  if (cudaMalloc(&b->d_state, bytes) != cudaSuccess) {
    set_error("batch state allocation of %zu bytes failed", bytes);
    return HPT_ENOMEM;
  }
  b->state_bytes = bytes;
  return HPT_OK;
}

hpt_status track_impl(hpt_batch_s* b, const int64_t* paths, const void* y0, const hpt_params& prm, void* x_out,
                      int32_t* status_out, int32_t* steps_out, cudaStream_t user) {
  const Problem q = plan(b, paths);
  b->rounds = 0;
  b->position_steps = 0;
  if (q.P == 0) return HPT_OK;
  hpt_status rc = ensure_state(b, q.total);
  if (rc) return rc;
  cudaStream_t st = b->own;
  cudaError_t e = cudaEventRecord(b->ev_in, user);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(st, b->ev_in, 0);
  if (e != cudaSuccess) return cuda_fail(e, "batch stream order");
  char* d = (char*)b->d_state;
  const hpt_paths S = state_of(b, q);
  // per-path variable offsets, per-system path offsets and counts, initial state
  std::vector<int32_t> np(b->nsys);
  for (int s = 0; s < b->nsys; ++s) np[s] = (int32_t)paths[s];
  e = cudaMemcpyAsync(d + q.o_pb, q.pb.data(), (size_t)b->nsys * 8, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d + q.o_np, np.data(), (size_t)b->nsys * 4, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_fail(e, "batch upload");
  for (int s = 0; s < b->nsys && e == cudaSuccess; ++s) {
    if (!paths[s]) continue;
    const int n = b->sys_n[s];
    fill_vofs_kernel<<<(unsigned)((paths[s] + 255) / 256), 256, 0, st>>>(paths[s], n, q.vb[s],
                                                                        (int64_t*)(d + q.o_vofs) + q.pb[s]);
    double tau0 = 0;
    hpt_get_info(b->sys[s], nullptr, nullptr, nullptr, prm.eps0, &tau0);
    e = launch_paths_init(b->sys[s], paths[s], (const char*)y0 + q.vb[s] * 16, tau0, prm,
                          sub_state(S, q.pb[s], q.vb[s]), st);
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_err, 0, 4, st);
  if (e == cudaSuccess) e = enqueue_compaction(b, q, S.status, HPT_PATH_ACTIVE, st);   // every path
  if (e != cudaSuccess) return cuda_fail(e, "batch init");
  // the round graph, captured again when the problem, the tuning or the
  // parameters changed (it holds them as launch arguments)
  const std::vector<int64_t> key(paths, paths + b->nsys);
  if (!b->exec || b->key_state != b->d_state || b->key_paths != key ||
      memcmp(&b->key_tune, &b->tune, sizeof(hpt_batch_tuning)) != 0 || !same_prm(b->key_prm, prm)) {
    if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
    cudaGraph_t g = nullptr;
    e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "batch capture");
    int32_t nk = 0;
    cudaError_t ec = enqueue_round(b, q, prm, st, &nk);
    e = cudaStreamEndCapture(st, &g);
    if (ec != cudaSuccess) { if (g) cudaGraphDestroy(g); return cuda_fail(ec, "batch round capture"); }
    if (e != cudaSuccess) return cuda_fail(e, "batch capture end");
    e = cudaGraphInstantiate(&b->exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) { b->exec = nullptr; return cuda_fail(e, "batch graph instantiate"); }
    b->key_state = b->d_state;
    b->key_paths = key;
    b->key_tune = b->tune;
    b->key_prm = prm;
    b->kernels_per_round = nk;
  }
  // rounds until no position is left or the step budget is spent
  e = cudaMemcpyAsync(b->h_ctl, d + q.o_ctl, kCtlWords * 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "batch init");
  const int K = b->tune.steps_per_round;
  int64_t steps = 0;
  while (b->h_ctl[0] > 0 && steps <= (int64_t)prm.max_steps + K) {
    b->position_steps += (int64_t)b->h_ctl[0] * K;
    e = cudaGraphLaunch(b->exec, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "batch round");
    ++b->rounds;
    steps += K;
  }
  // outputs, then the FP64 polish per system
  int32_t* done = (int32_t*)(d + q.o_done);
  float* last = (float*)(d + q.o_last);
  for (int s = 0; s < b->nsys && e == cudaSuccess; ++s) {
    if (!paths[s]) continue;
    e = launch_finish_track(b->sys[s], paths[s], sub_state(S, q.pb[s], q.vb[s]), (char*)x_out + q.vb[s] * 16,
                            status_out ? status_out + q.pb[s] : nullptr, steps_out ? steps_out + q.pb[s] : nullptr,
                            done + q.pb[s], st);
  }
  if (e != cudaSuccess) return cuda_fail(e, "batch output");
  // FP64 Newton polish of the converged paths of every system at once:
  // each iteration compacts the paths still to polish (done == 0), then per
  // shape bucket evaluates (FP64) and updates them
  int32_t* ctl = (int32_t*)(d + q.o_ctl);
  PathMap pm;
  pm.list = (const int64_t*)(d + q.o_list);
  pm.tile_sys = (const int32_t*)(d + q.o_tsys);
  pm.sys_n = b->d_sys_n;
  pm.vofs = (const int64_t*)(d + q.o_vofs);
  pm.nmax = b->nmax;
  e = cudaMemsetAsync(last, 0, (size_t)q.P * sizeof(float), st);
  if (e != cudaSuccess) return cuda_fail(e, "batch polish init");
  for (int it = 0; it < prm.polish_iters; ++it) {
    e = enqueue_compaction(b, q, done, 0, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->h_ctl, ctl, kCtlWords * 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "batch polish compaction");
    if (b->h_ctl[0] == 0) break;
    for (int bk = 0; bk < kBuckets && e == cudaSuccess; ++bk) {
      if (!q.cap_bucket[bk]) continue;
      pm.pos_begin = ctl + 1 + bk;
      pm.npos = ctl + 1 + kBuckets + bk;
      const int sh = bk < 2 ? bk : 2;   // FP64: n <= 8, <= 16, <= 32 lane groups
      // evaluation sized for the bucket's variables (n <= 8, 16, 24, 32)
      const int esh = bk < 2 ? bk : (bk == 2 ? kEval24 : 2);
      e = launch_eval_fp64_map(esh, b->d_f64, q.cap_bucket[bk], x_out, nullptr, pm, d + q.o_ext, st);
      if (e == cudaSuccess)
        e = launch_newton_map(sh, q.cap_bucket[bk], d + q.o_ext, x_out, done, last, prm.polish_tol, pm, st);
    }
    if (e != cudaSuccess) return cuda_fail(e, "batch polish");
  }
  e = cudaEventRecord(b->ev_out, st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(user, b->ev_out, 0);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "batch track");
  int32_t herr = 0;
  e = cudaMemcpy(&herr, b->d_err, 4, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "batch error flag");
  if (herr) { set_error("a bounded device-side wait gave up"); return HPT_ETIMEOUT; }
  return HPT_OK;
}

hpt_status check_batch(hpt_batch b) {
  if (!b) { set_error("NULL batch"); return HPT_EINVAL; }
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != b->device) {
    set_error("the batch belongs to device %d, current device is %d", b->device, dev);
    return HPT_EINVAL;
  }
  return HPT_OK;
}

hpt_status check_paths(hpt_batch b, const int64_t* paths, const void* y0, const void* x_out) {
  if (!paths) { set_error("paths is NULL"); return HPT_EINVAL; }
  int64_t tot = 0;
  for (int s = 0; s < b->nsys; ++s) {
    if (paths[s] < 0 || paths[s] > ((int64_t)1 << 30)) { set_error("paths[%d] out of range", s); return HPT_EINVAL; }
    tot += paths[s];
  }
  if (tot > ((int64_t)1 << 31) - (int64_t)b->nsys * 128) { set_error("too many paths"); return HPT_EINVAL; }
  if (tot > 0 && (!y0 || !x_out)) { set_error("y0 or x_out is NULL"); return HPT_EINVAL; }
  return HPT_OK;
}

}  // namespace
}  // namespace hpt

using namespace hpt;

extern "C" {

hpt_status hpt_batch_create(int32_t nsys, const hpt_system* systems, hpt_batch* out) {
  if (!out) { set_error("out is NULL"); return HPT_EINVAL; }
  *out = nullptr;
  if (nsys < 1 || !systems) { set_error("need nsys >= 1 systems"); return HPT_EINVAL; }
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) { set_error("no current device"); return HPT_ECUDA; }
  for (int s = 0; s < nsys; ++s) {
    if (!systems[s]) { set_error("system %d is NULL", s); return HPT_EINVAL; }
    if (systems[s]->prec != HPT_MIXED) { set_error("system %d is not HPT_MIXED", s); return HPT_ENOTSUP; }
    if (systems[s]->proj) { set_error("system %d is projective (batches hold affine systems)", s); return HPT_ENOTSUP; }
    if (systems[s]->device != dev) { set_error("system %d belongs to another device", s); return HPT_EINVAL; }
  }
  hpt_batch b = new hpt_batch_s();
  b->device = dev;
  b->nsys = nsys;
  b->sys.assign(systems, systems + nsys);
  std::vector<MixedSys> tab(nsys);
  std::vector<double> cost(nsys);
  int64_t chunk_total = 0;
  MixedSys& mx = b->maxs;
  memset(&mx, 0, sizeof(mx));
  for (int s = 0; s < nsys; ++s) {
    const hpt_system h = systems[s];
    tab[s] = mixed_sys_of(h);
    tab[s].chunk_off = chunk_total;
    chunk_total += (int64_t)h->n * h->ml.chunk_bytes;
    b->sys_n.push_back(h->n);
    b->bucket.push_back(bucket_of(h->n));
    mx.n = std::max(mx.n, h->n);
    mx.MP = std::max(mx.MP, h->ml.MP);
    mx.KX = std::max(mx.KX, h->ml.KX);
    mx.NJ = std::max(mx.NJ, h->ml.NJ);
    mx.KC = std::max(mx.KC, h->ml.KC);
    mx.chunk_bytes = std::max(mx.chunk_bytes, h->ml.chunk_bytes);
    mx.off_bhi = std::max(mx.off_bhi, h->ml.off_bhi);     // the largest exponent part
    mx.off_aint = std::max(mx.off_aint, h->ml.off_aint);   // nonzero: some system has large exponents
    mx.off_bigm = std::max(mx.off_bigm, h->ml.off_bigm);
    mx.tcols1 = std::max(mx.tcols1, tab[s].tcols1);   // per system: its own W and J widths
    mx.tcols2 = std::max(mx.tcols2, tab[s].tcols2);
    b->tmem_cols = std::max(b->tmem_cols, h->ml.tmem_cols);
    b->nmax = std::max(b->nmax, h->n);
    // evaluation work of one tile: n equations x (exponent + coefficient GEMM + exp)
    cost[s] = (double)h->n * (h->ml.MP * (double)h->ml.KX + 3.0 * h->ml.NJ * h->ml.KC + 8.0 * h->ml.MP);
  }
  b->redo_shape = solve_shape_of(b->nmax);
  b->order.resize(nsys);
  std::iota(b->order.begin(), b->order.end(), 0);
  std::stable_sort(b->order.begin(), b->order.end(), [&](int x, int y) {
    if (b->bucket[x] != b->bucket[y]) return b->bucket[x] < b->bucket[y];
    return cost[x] > cost[y];
  });
  for (int k = 0; k < kBuckets; ++k) b->span.first[k] = b->span.last[k] = -1;
  for (int i = 0; i < nsys; ++i) {
    const int k = b->bucket[b->order[i]];
    if (b->span.first[k] < 0) b->span.first[k] = i;
    b->span.last[k] = i;
  }
  b->tune.eval_ctas_per_sm = eval_mixed_max_ctas(b->tmem_cols);
  cudaError_t e = cudaMalloc(&b->d_chunks, (size_t)chunk_total);
  for (int s = 0; s < nsys && e == cudaSuccess; ++s)
    e = cudaMemcpy(b->d_chunks + tab[s].chunk_off, systems[s]->d_chunks, (size_t)systems[s]->n * systems[s]->ml.chunk_bytes,
                   cudaMemcpyDeviceToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_tab, sizeof(MixedSys) * nsys);
  if (e == cudaSuccess) e = cudaMemcpy(b->d_tab, tab.data(), sizeof(MixedSys) * nsys, cudaMemcpyHostToDevice);
  std::vector<Fp64Sys> f64(nsys);
  for (int s = 0; s < nsys; ++s) f64[s] = fp64_sys_of(systems[s]);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_f64, sizeof(Fp64Sys) * nsys);
  if (e == cudaSuccess) e = cudaMemcpy(b->d_f64, f64.data(), sizeof(Fp64Sys) * nsys, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_sys_n, 4 * nsys);
  if (e == cudaSuccess) e = cudaMemcpy(b->d_sys_n, b->sys_n.data(), 4 * nsys, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_order, 4 * nsys);
  if (e == cudaSuccess) e = cudaMemcpy(b->d_order, b->order.data(), 4 * nsys, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_err, 4);
  if (e == cudaSuccess) e = cudaMemset(b->d_err, 0, 4);
  if (e == cudaSuccess) e = cudaMallocHost(&b->h_ctl, kCtlWords * 4);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->own, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    hpt_status rc = cuda_fail(e, "batch create");
    hpt_batch_destroy(b);
    return rc;
  }
  *out = b;
  return HPT_OK;
}

hpt_status hpt_batch_destroy(hpt_batch b) {
  if (!b) return HPT_EINVAL;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(b->device);
  if (b->own) cudaStreamSynchronize(b->own);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  cudaFree(b->d_chunks);
  cudaFree(b->d_tab);
  cudaFree(b->d_f64);
  cudaFree(b->d_sys_n);
  cudaFree(b->d_order);
  cudaFree(b->d_err);
  cudaFree(b->d_state);
  if (b->h_ctl) cudaFreeHost(b->h_ctl);
  if (b->own) cudaStreamDestroy(b->own);
  if (b->ev_in) cudaEventDestroy(b->ev_in);
  if (b->ev_out) cudaEventDestroy(b->ev_out);
  cudaSetDevice(prev);
  delete b;
  return HPT_OK;
}

hpt_status hpt_batch_get_tuning(hpt_batch b, hpt_batch_tuning* t) {
  if (!b || !t) { set_error("NULL argument"); return HPT_EINVAL; }
  *t = b->tune;
  return HPT_OK;
}

hpt_status hpt_batch_set_tuning(hpt_batch b, const hpt_batch_tuning* t) {
  if (!b || !t) { set_error("NULL argument"); return HPT_EINVAL; }
  if (t->steps_per_round < 1 || t->steps_per_round > 256 || t->eval_ctas_per_sm < 1 || t->eval_ctas_per_sm > 2 ||
      (t->solve_lanes_n17_24 != 8 && t->solve_lanes_n17_24 != 32)) {
    set_error("tuning out of range");
    return HPT_EINVAL;
  }
  b->tune = *t;
  b->tune.eval_ctas_per_sm = std::min(t->eval_ctas_per_sm, eval_mixed_max_ctas(b->tmem_cols));
  return HPT_OK;
}

hpt_status hpt_batch_track(hpt_batch b, const int64_t* paths, const void* y0, const hpt_params* prm, void* x_out,
                           int32_t* status_out, int32_t* steps_out, void* stream) {
  hpt_status rc = check_batch(b);
  if (rc) return rc;
  if ((rc = check_params(prm))) return rc;
  if ((rc = check_paths(b, paths, y0, x_out))) return rc;
  return track_impl(b, paths, y0, *prm, x_out, status_out, steps_out, (cudaStream_t)stream);
}

hpt_status hpt_batch_autotune(hpt_batch b, const int64_t* paths, const void* y0, const hpt_params* prm,
                              void* x_out, void* stream, hpt_batch_tuning* best, hpt_batch_tuning* cand,
                              double* ms, int32_t* ncand) {
  hpt_status rc = check_batch(b);
  if (rc) return rc;
  if ((rc = check_params(prm))) return rc;
  if ((rc = check_paths(b, paths, y0, x_out))) return rc;
  const int cap = ncand ? *ncand : 0;
  int count = 0;
  hpt_batch_tuning win = b->tune;
  double win_ms = -1;
  // times one candidate; keeps it if it is the fastest so far
  auto trial = [&](const hpt_batch_tuning& t) -> hpt_status {
    b->tune = t;
    const auto t0 = std::chrono::steady_clock::now();
    hpt_status r = track_impl(b, paths, y0, *prm, x_out, nullptr, nullptr, (cudaStream_t)stream);
    const auto t1 = std::chrono::steady_clock::now();
    if (r) return r;
    const double el = std::chrono::duration<double, std::milli>(t1 - t0).count();
    if (count < cap) {
      if (cand) cand[count] = t;
      if (ms) ms[count] = el;
    }
    ++count;
    if (win_ms < 0 || el < win_ms) { win_ms = el; win = t; }
    return HPT_OK;
  };
  const hpt_batch_tuning start = b->tune;
  const int max_ctas = eval_mixed_max_ctas(b->tmem_cols);
  hpt_batch_tuning t = start;
  for (int lanes : {8, 32}) {
    t.solve_lanes_n17_24 = lanes;
    if ((rc = trial(t))) { b->tune = start; return rc; }
  }
  t = win;
  for (int c = 1; c <= max_ctas; ++c) {
    if (c == win.eval_ctas_per_sm) continue;
    t.eval_ctas_per_sm = c;
    if ((rc = trial(t))) { b->tune = start; return rc; }
  }
  t = win;
  for (int K : {2, 4, 8, 16, 32}) {
    if (K == win.steps_per_round) continue;
    t.steps_per_round = K;
    if ((rc = trial(t))) { b->tune = start; return rc; }
  }
  b->tune = win;
  if (best) *best = win;
  if (ncand) *ncand = std::min(count, cap);
  return HPT_OK;
}

hpt_status hpt_batch_stats(hpt_batch b, int64_t* rounds, int64_t* position_steps, int32_t* kernels_per_round) {
  if (!b) { set_error("NULL batch"); return HPT_EINVAL; }
  if (rounds) *rounds = b->rounds;
  if (position_steps) *position_steps = b->position_steps;
  if (kernels_per_round) *kernels_per_round = b->kernels_per_round;
  return HPT_OK;
}

}  // extern "C"
