// Pipelined mixed-precision evaluation for the step of one system: the same
// arithmetic as eval_mixed_kernel (Algorithm 2, Section 5: exponent GEMM on
// the tensor cores, complex exponential, coefficient GEMM; op. 1 and the
// exponential through the shared log_coords / cexp_split8, the GEMMs with the
// same instruction shapes, operands and order, so both kernels give the same
// bits), organised so that the tensor core, the special-function units and
// the stores of different equations overlap.  One persistent CTA per SM
// works through a contiguous range of (tile, equation) units, tiles of 128
// points (point r = tensor-memory lane r), with warp roles that hand buffers
// to one another through mbarriers:
//   exp warps   (warps 0-15, four warpgroups over the 128 lanes, splitting the
//               monomial columns in chunks of 8): read the exponent
//               accumulator W of unit i from tensor memory, form E and write
//               its BF16 hi/lo parts as the A operand of the coefficient GEMM;
//               at the first unit of a tile they also form the log
//               coordinates (op. 1) of the next tile, a quarter of the
//               variables per warpgroup;
//   drain warps (warps 16-19, one per lane quarter): read the coefficient
//               accumulator J of unit i from tensor memory and store the row
//               [D_z h_k | D_tau h_k | h_k] of every point to the scratch;
//   MMA warp    (warp 20; the whole warp runs the issue loop, one elected lane
//               issues each MMA and commit): issues the exponent GEMMs of
//               up to kWBuf - 1 units ahead of the coefficient GEMM of unit
//               i, so the tensor core works ahead while the exp warps work
//               on i;
//   load warp   (warp 21, one thread): bulk-copies the constant image of
//               each unit's equation (exponent operand, t-exponents, B_k hi/lo)
//               into a ring of kCBuf buffers, so that a copy starts kCBuf - 1
//               units ahead of the exponent GEMM that reads it.
// W is a ring of kWBuf tensor-memory buffers, E a ring of kEBuf shared-memory
// buffers and J a ring of kJBuf tensor-memory buffers; the log coordinates of
// two tiles are kept.  Every mbarrier wait is bounded (about two seconds);
// a wait that gives up raises the device error flag and the CTA winds down
// after the copies and MMAs it issued have landed.
#include <algorithm>

#include "hpt_internal.h"
#include "hpt_tc.cuh"

namespace hpt {
namespace {

constexpr int kExpWarps = 16;
constexpr int kDrainWarps = 4;
constexpr int kMmaWarp = kExpWarps + kDrainWarps;
constexpr int kLoadWarp = kMmaWarp + 1;
constexpr int kPipeThreads = (kLoadWarp + 1) * 32;   // 704
constexpr int kCBuf = 4;                              // constant-image ring
constexpr int kWBuf = 3;                              // exponent accumulators W in tensor memory
constexpr int kEBuf = 3;                              // coefficient-GEMM A operands E in shared memory
constexpr int kJBuf = 2;                              // coefficient accumulators J in tensor memory

struct PipeArgs {
  MixedSys sys;
  int64_t p;
  int ntiles;
  int tmem_cols;
  // shared-memory carve-up (bytes from the 1024-aligned base)
  int s_z[2];        // log coordinates of a tile: Re (128 x KX bf16), Im, tau2[128], fixed angles
  int z_im, z_tau, z_q;   // offsets inside a log-coordinate buffer (z_q: [j][128] uint32)
  int s_e[kEBuf];    // coefficient-GEMM A operand: hi (128 x KC bf16), then lo
  int e_lo;
  int s_c[kCBuf];    // constant images
  int s_bar;
};

// Barriers.  One "coefficient GEMM of unit i done" ring (slot i % kDone)
// stands for three events: J of unit i full (drain), E buffer of unit i free
// (exp warps, kEBuf units later), constant buffer of unit i free (loader,
// kCBuf units later); every waiter is at most one completion behind its slot.
// The exp warps' "E full" also frees their W buffer: the MMA warp issues the
// exponent GEMM into it only after it has waited for that arrival.
constexpr int kDone = kCBuf;
static_assert(kDone >= kEBuf && kDone >= kJBuf, "done ring");
enum { B_CFULL = 0, B_DONE = B_CFULL + kCBuf, B_ZFULL = B_DONE + kDone, B_ZEMPTY = B_ZFULL + 2,
       B_WFULL = B_ZEMPTY + 2, B_EFULL = B_WFULL + kWBuf, B_JEMPTY = B_EFULL + kEBuf, B_COUNT = B_JEMPTY + kJBuf };

__global__ void __launch_bounds__(kPipeThreads, 1)
eval_pipe_kernel(PipeArgs P, const float2* __restrict__ y, const double* __restrict__ tau_in,
                 const uint8_t* __restrict__ chunks, float2* __restrict__ ext, int32_t* __restrict__ err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* sm = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = (uint64_t*)(sm + P.s_bar);
  uint32_t* tslot = (uint32_t*)(sm + P.s_bar + B_COUNT * 8);
  volatile int* sAbort = (volatile int*)(sm + P.s_bar + B_COUNT * 8 + 4);
  const MixedSys& S = P.sys;
  const int n = S.n, ne = S.ne;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  // this CTA's units [u0, u1) of the tile-major sequence of (tile, equation)
  const int64_t units = (int64_t)P.ntiles * ne;
  const int64_t u0 = (int64_t)blockIdx.x * units / (int64_t)gridDim.x;
  const int64_t u1 = ((int64_t)blockIdx.x + 1) * units / (int64_t)gridDim.x;
  const int U = (int)(u1 - u0);
  if (U <= 0) return;
  const int t_first = (int)(u0 / ne);
  const int t_last = (int)((u1 - 1) / ne);
  const int k_first = (int)(u0 - (int64_t)t_first * ne);
  // Unit i is equation k of local tile lt; every role walks the units in
  // order, so it steps (k, lt) along instead of dividing.
  struct Unit {
    int i, k, lt;
  };
  auto next_unit = [&](Unit u) {
    ++u.i;
    if (++u.k == ne) {
      u.k = 0;
      ++u.lt;
    }
    return u;
  };
  const Unit first_unit = {0, k_first, 0};
  auto first_of_tile = [&](const Unit& u) { return u.i == 0 || u.k == 0; };
  auto last_of_tile = [&](const Unit& u) { return u.i == U - 1 || u.k == ne - 1; };
  auto bar = [&](int b) { return su32(&bars[b]); };
  auto wait = [&](int b, int use) -> bool {   // the use-th completion of barrier b
    if (*sAbort) return false;
    if (mbar_wait(bar(b), (uint32_t)use & 1u)) return true;
    *sAbort = 1;
    return false;
  };

  if (tid == 0) {
    for (int q = 0; q < kCBuf; ++q) mbar_init(bar(B_CFULL + q), 1);
    for (int q = 0; q < kDone; ++q) mbar_init(bar(B_DONE + q), 1);
    for (int q = 0; q < 2; ++q) {
      mbar_init(bar(B_ZFULL + q), kExpWarps);
      mbar_init(bar(B_ZEMPTY + q), 1);
    }
    for (int q = 0; q < kWBuf; ++q) mbar_init(bar(B_WFULL + q), 1);
    for (int q = 0; q < kEBuf; ++q) mbar_init(bar(B_EFULL + q), kExpWarps);
    for (int q = 0; q < kJBuf; ++q) mbar_init(bar(B_JEMPTY + q), kDrainWarps);
    *sAbort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == kMmaWarp) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tslot)),
                 "r"(P.tmem_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = *tslot;
  // tensor-memory columns: the W ring (Re MP, Im MP each), then the J ring
  auto tw_col = [&](int b) { return tbase + (uint32_t)(b * 2 * S.MP); };
  // unit i's buffer in a ring of R, and the completion of that buffer's
  // barrier that unit i waits for: its (i / R)-th as "full", the (i / R - 1)-th
  // (unit i - R's) as "empty"
  auto ring = [](int i, int R) { return i % R; };
  auto use = [](int i, int R) { return i / R; };
  // buffer offsets by selection (an indexed kernel-parameter array would be
  // copied to local memory)
  auto zoff = [&](int b) { return b ? P.s_z[1] : P.s_z[0]; };
  auto eoff = [&](int e) {
    int o = P.s_e[0];
#pragma unroll
    for (int q = 1; q < kEBuf; ++q) o = e == q ? P.s_e[q] : o;
    return o;
  };
  auto coff = [&](int c) {
    int o = P.s_c[0];
#pragma unroll
    for (int q = 1; q < kCBuf; ++q) o = c == q ? P.s_c[q] : o;
    return o;
  };
  auto tj_col = [&](int b) { return tbase + (uint32_t)(kWBuf * 2 * S.MP + b * S.NJ); };

  if (warp < kExpWarps) {
    // ---------------- exp warps ----------------
    const int wg = warp >> 2;
    const int row = (warp & 3) * 32 + lane;
    const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
    // op. 1 for local tile lt: log coordinates, three-way BF16 split; this
    // warpgroup takes the variables wg, wg + 4, ...
    auto prep_z = [&](int lt) -> bool {
      if (lt >= 2 && !wait(B_ZEMPTY + (lt & 1), (lt >> 1) - 1)) return false;
      uint8_t* zre = sm + zoff(lt & 1);
      uint8_t* zim = zre + P.z_im;
      const int64_t pos = (int64_t)(t_first + lt) * 128 + row;
      const bool live = pos < P.p;
      if (wg == 0) {
        const double tau = live ? tau_in[pos] : 0.0;
        ((float*)(zre + P.z_tau))[row] = (float)(tau * (double)S.inv_D * 1.4426950408889634);   // (tau/D) log2(e)
      }
      for (int j = wg; j < n; j += 4) {
        const float2 v = live ? y[(size_t)pos * n + j] : make_float2(1.f, 0.f);
        float rem_r, rem_i;
        log_coords(v, rem_r, rem_i);
        if (S.off_aint) ((uint32_t*)(zre + P.z_q))[j * 128 + row] = fixed_angle(rem_i);
#pragma unroll
        for (int s = 0; s < 3; ++s) {
          const uint16_t hr = bf16_rn(rem_r), hi = bf16_rn(rem_i);
          *(uint16_t*)(zre + canon(row, s * n + j, S.KX)) = hr;
          *(uint16_t*)(zim + canon(row, s * n + j, S.KX)) = hi;
          rem_r -= bf16_f(hr);
          rem_i -= bf16_f(hi);
        }
      }
      for (int q = 3 * n + wg; q < S.KX; q += 4) {
        *(uint16_t*)(zre + canon(row, q, S.KX)) = 0;
        *(uint16_t*)(zim + canon(row, q, S.KX)) = 0;
      }
      proxy_fence();
      __syncwarp();
      if (lane == 0) mbar_arrive(bar(B_ZFULL + (lt & 1)));
      return true;
    };
    float tau2 = 0.f;
    const uint32_t* zq = nullptr;   // this point's fixed angles (large exponents)
    for (Unit u = first_unit; u.i < U; u = next_unit(u)) {
      const int i = u.i, w = ring(i, kWBuf), e = ring(i, kEBuf), lt = u.lt;
      if (first_of_tile(u)) {
        if (i == 0 && !prep_z(0)) break;
        if (t_first + lt + 1 <= t_last && !prep_z(lt + 1)) break;   // the next tile, one tile ahead
        if (!wait(B_ZFULL + (lt & 1), lt >> 1)) break;
        tau2 = ((const float*)(sm + zoff(lt & 1) + P.z_tau))[row];
        zq = (const uint32_t*)(sm + zoff(lt & 1) + P.z_q) + row;
      }
      if (!wait(B_WFULL + w, use(i, kWBuf))) break;
      if (i >= kEBuf && !wait(B_DONE + ring(i - kEBuf, kDone), use(i - kEBuf, kDone))) break;
      tc_fence_after();
      // the t-exponents (and large-exponent tables) of unit i's equation,
      // read through L1 from its constant image in global memory
      const uint8_t* cg = chunks + (size_t)u.k * S.chunk_bytes;
      const float* texp = (const float*)(cg + S.off_texp);
      uint8_t* eh = sm + eoff(e);
      uint8_t* el = eh + P.e_lo;
      for (int c0 = 8 * wg; c0 < S.MP; c0 += 8 * 4) {
        uint32_t wre[8], wim[8];
        tmem_ld8(tw_col(w) + lane_base + c0, wre);
        tmem_ld8(tw_col(w) + lane_base + S.MP + c0, wim);
        tmem_wait_ld();
        uint4 hre, lre, him, lim;
        const uint32_t big8 = S.off_bigm ? (((const uint32_t*)(cg + S.off_bigm))[c0 >> 5] >> (c0 & 31)) & 0xffu : 0u;
        cexp_split8(wre, wim, texp + c0, tau2, big8, (const int16_t*)(cg + S.off_aint) + c0 * n, zq, n, hre, lre,
                    him, lim);
        // Re E at K = c0.., Im E at K = MP + c0..; 8 values = one core column
        *(uint4*)(eh + canon(row, c0, S.KC)) = hre;
        *(uint4*)(el + canon(row, c0, S.KC)) = lre;
        *(uint4*)(eh + canon(row, S.MP + c0, S.KC)) = him;
        *(uint4*)(el + canon(row, S.MP + c0, S.KC)) = lim;
      }
      tc_fence_before();
      proxy_fence();
      __syncwarp();
      if (lane == 0) mbar_arrive(bar(B_EFULL + e));   // E full, W buffer free
    }
  } else if (warp < kMmaWarp) {
    // ---------------- drain warps ----------------
    const int row = (warp & 3) * 32 + lane;
    const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
    for (Unit u = first_unit; u.i < U; u = next_unit(u)) {
      const int i = u.i, b = ring(i, kJBuf), lt = u.lt, k = u.k;
      if (!wait(B_DONE + ring(i, kDone), use(i, kDone))) break;
      tc_fence_after();
      const int64_t pos = (int64_t)(t_first + lt) * 128 + row;
      const bool live = pos < P.p;
      float2* erow = ext + ext_index(pos, k, 0, n);
      for (int c0 = 0; c0 < 2 * (n + 2); c0 += 8) {
        uint32_t jr[8];
        tmem_ld8(tj_col(b) + lane_base + c0, jr);
        tmem_wait_ld();
        if (live) {
#pragma unroll
          for (int v = 0; v < 4; ++v) {
            const int u = c0 / 2 + v;
            if (u < n + 2) erow[(size_t)u * 128] = make_float2(__uint_as_float(jr[2 * v]), __uint_as_float(jr[2 * v + 1]));
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(bar(B_JEMPTY + b));
    }
  } else if (warp == kMmaWarp) {
    // ---------------- MMA issuer: the whole warp runs the loop, one elected
    // lane issues each MMA and commit ----------------
    {
      // a failed (timed-out) wait in any lane stops every lane: elect.sync
      // needs the whole warp
      auto waitw = [&](int bb, int uu) { return __all_sync(0xffffffffu, wait(bb, uu)); };
      const uint32_t idx_x = idesc_bf16(128, S.MP), sbo_x = S.KX * 16;
      const uint32_t idx_c = idesc_bf16(128, S.NJ), sbo_c = S.KC * 16;
      int last_exp = -1, last_coef = -1;
      auto issue_exp = [&](const Unit& u) -> bool {
        const int i = u.i, w = ring(i, kWBuf), c = ring(i, kCBuf), lt = u.lt;
        if (first_of_tile(u) && !waitw(B_ZFULL + (lt & 1), lt >> 1)) return false;
        if (!waitw(B_CFULL + c, use(i, kCBuf))) return false;
        tc_fence_after();
        const uint32_t cb = su32(sm + coff(c));
        const uint32_t zre = su32(sm + zoff(lt & 1)), zim = zre + (uint32_t)P.z_im;
        const uint32_t tw = tw_col(w);
        // a K-slice of 256 bytes adds 16 to a descriptor's address field
        const uint64_t bd = smem_desc(cb + S.off_bexp, 128, sbo_x);
        const uint64_t ar = smem_desc(zre, 128, sbo_x), ai = smem_desc(zim, 128, sbo_x);
        for (int s = 0; s < S.KX / 16; ++s) {
          mma_bf16_w(tw, ar + 16 * s, bd + 16 * s, idx_x, s > 0);
          mma_bf16_w(tw + S.MP, ai + 16 * s, bd + 16 * s, idx_x, s > 0);
        }
        mma_commit_w(bar(B_WFULL + w));
        if (last_of_tile(u)) mma_commit_w(bar(B_ZEMPTY + (lt & 1)));
        last_exp = i;
        return true;
      };
      // the exponent GEMMs run kWBuf - 1 units ahead of the coefficient GEMM
      // (the exp warps prepare a tile's log coordinates a tile ahead)
      Unit ahead = first_unit;
      bool ok = true;
      for (int q = 0; ok && q < kWBuf - 1 && ahead.i < U; ++q, ahead = next_unit(ahead)) ok = issue_exp(ahead);
      for (Unit u = first_unit; ok && u.i < U; u = next_unit(u)) {
        const int i = u.i, e = ring(i, kEBuf), b = ring(i, kJBuf), c = ring(i, kCBuf);
        if (ahead.i < U) {
          if (!(ok = issue_exp(ahead))) break;
          ahead = next_unit(ahead);
        }
        if (!waitw(B_EFULL + e, use(i, kEBuf))) break;
        if (i >= kJBuf && !waitw(B_JEMPTY + b, use(i, kJBuf) - 1)) break;
        tc_fence_after();
        const uint32_t cb = su32(sm + coff(c));
        const uint32_t ah0 = su32(sm + eoff(e)), al0 = ah0 + (uint32_t)P.e_lo;
        const uint32_t tj = tj_col(b);
        coef_gemm(tj, smem_desc(ah0, 128, sbo_c), smem_desc(al0, 128, sbo_c), smem_desc(cb + S.off_bhi, 128, sbo_c),
                  smem_desc(cb + S.off_blo, 128, sbo_c), idx_c, S.KC / 16);
        mma_commit_w(bar(B_DONE + ring(i, kDone)));
        last_coef = i;
      }
      if (*sAbort) {
        // let the MMAs issued land before the CTA's memory goes away
        if (last_coef >= 0)
          mbar_wait(bar(B_DONE + ring(last_coef, kDone)), (uint32_t)use(last_coef, kDone) & 1u);
        if (last_exp > last_coef)
          mbar_wait(bar(B_WFULL + ring(last_exp, kWBuf)), (uint32_t)use(last_exp, kWBuf) & 1u);
      }
    }
  } else {
    // ---------------- constant loads ----------------
    if (lane == 0) {
      int issued = 0;
      for (Unit u = first_unit; u.i < U; u = next_unit(u)) {
        const int i = u.i, c = ring(i, kCBuf);
        if (i >= kCBuf && !wait(B_DONE + ring(i - kCBuf, kDone), use(i - kCBuf, kDone))) break;
        bulk_load(su32(sm + coff(c)), chunks + (size_t)u.k * S.chunk_bytes, S.chunk_bytes, bar(B_CFULL + c));
        issued = i + 1;
      }
      if (*sAbort) {
        // let the copies issued land
        for (int i = issued > kCBuf ? issued - kCBuf : 0; i < issued; ++i)
          mbar_wait(bar(B_CFULL + ring(i, kCBuf)), (uint32_t)use(i, kCBuf) & 1u);
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  if (*sAbort && tid == 0) atomicExch(err, 1);
  if (warp == kMmaWarp) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(P.tmem_cols));
  }
}

}  // namespace

// Shared memory the pipelined kernel needs for these shapes (0: it does not
// serve them).
int eval_pipe_smem(const MixedSys& s) {
  // the W and J rings in the 512 tensor-memory columns of the SM
  if (s.n > 16 || s.ne != s.n || kWBuf * 2 * s.MP + kJBuf * s.NJ > 512) return 0;
  auto r1k = [](int v) { return (v + 1023) / 1024 * 1024; };
  const int z = r1k(2 * 128 * s.KX * 2 + 128 * 4 + (s.off_aint ? 128 * s.n * 4 : 0));
  const int e = r1k(2 * 128 * s.KC * 2);
  const int c = r1k(s.chunk_bytes);
  return 2 * z + kEBuf * e + kCBuf * c + 1024 + 1024;   // barriers, slack for aligning the base
}

cudaError_t launch_eval_pipe(hpt_system prof, const MixedSys& s, int64_t p, const uint8_t* chunks, const void* y,
                             const double* tau, void* ext, int32_t* err, int num_sms, cudaStream_t st) {
  const int smem = eval_pipe_smem(s);
  if (!smem) return cudaErrorInvalidValue;
  PipeArgs a{};
  a.sys = s;
  a.p = p;
  const int64_t ntiles = (p + 127) / 128;
  if (ntiles > 0x7fffffff) return cudaErrorInvalidValue;
  a.ntiles = (int)ntiles;
  int cols = kWBuf * 2 * s.MP + kJBuf * s.NJ, t = 32;
  while (t < cols) t *= 2;
  if (t > 512) return cudaErrorInvalidValue;
  a.tmem_cols = t;
  auto r1k = [](int v) { return (v + 1023) / 1024 * 1024; };
  int off = 0;
  const int zb = r1k(2 * 128 * s.KX * 2 + 128 * 4 + (s.off_aint ? 128 * s.n * 4 : 0));
  const int eb = r1k(2 * 128 * s.KC * 2), cbb = r1k(s.chunk_bytes);
  a.z_im = 128 * s.KX * 2;
  a.z_tau = 2 * 128 * s.KX * 2;
  a.z_q = a.z_tau + 128 * 4;
  a.e_lo = 128 * s.KC * 2;
  for (int q = 0; q < 2; ++q) { a.s_z[q] = off; off += zb; }
  for (int q = 0; q < kEBuf; ++q) { a.s_e[q] = off; off += eb; }
  for (int q = 0; q < kCBuf; ++q) { a.s_c[q] = off; off += cbb; }
  a.s_bar = off;
  cudaError_t e = cudaFuncSetAttribute(eval_pipe_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  const int64_t units = ntiles * s.ne;
  const int64_t grid = std::min<int64_t>(units, num_sms);
  if (grid < 1) return cudaSuccess;
  int pi = prof_begin(prof, "eval_pipe_tc", st);
  eval_pipe_kernel<<<(unsigned)grid, kPipeThreads, smem, st>>>(a, (const float2*)y, tau, chunks, (float2*)ext, err);
  prof_end(prof, pi, st);
  return cudaGetLastError();
}

}  // namespace hpt
