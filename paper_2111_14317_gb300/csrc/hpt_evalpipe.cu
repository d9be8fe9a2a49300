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
//               variables per warpgroup (the four drain warps alone took
//               three times as long);
//   drain warps (warps 16-19, one per lane quarter): read the coefficient
//               accumulator J of unit i from tensor memory and store the row
//               [D_z h_k | D_tau h_k | h_k] of every point to the scratch;
//   MMA issuers (warps 20-23, one per SM sub-partition; each walks its loop
//               as a whole warp and lane 0 issues): XR and XI issue the Re
//               and Im halves of the exponent GEMM up to kWBuf units ahead,
//               CH and CL the E_hi and E_lo parts of the coefficient GEMM
//               into their own column groups of J, so that four MMAs are in
//               issue at once (an MMA holds its issuing thread for about a
//               hundred cycles, whatever its N);
//   load warp   (warp 24, one thread): bulk-copies the constant image of
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
constexpr int kXrWarp = kExpWarps + kDrainWarps;      // exponent GEMM, Re half
constexpr int kXiWarp = kXrWarp + 1;                  // exponent GEMM, Im half
constexpr int kChWarp = kXrWarp + 2;                  // coefficient GEMM, E_hi part
constexpr int kClWarp = kXrWarp + 3;                  // coefficient GEMM, E_lo part
constexpr int kLoadWarp = kXrWarp + 4;
constexpr int kPipeThreads = (kLoadWarp + 1) * 32;   // 800
static_assert(kChWarp % 4 != kClWarp % 4 && kXrWarp % 4 != kXiWarp % 4, "issuers on separate sub-partitions");
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
// stands for three events: J of unit i full (drain), constant buffer of
// unit i free (loader, kCBuf units later) and E buffer of unit i free (the
// exponent-GEMM issuers, kEBuf units later, before they issue the GEMM whose
// W the exp warps wait for); every waiter is at most one completion behind
// its slot.  The exp warps' "E full" also frees their W buffer: the
// coefficient GEMM of that unit waits for it, so "done" of unit i - kEBuf
// tells the exponent-GEMM issuers that W buffer i - kWBuf is free as well.
constexpr int kDone = kCBuf;
static_assert(kDone >= kEBuf && kDone >= kJBuf, "done ring");
static_assert(kWBuf == kEBuf, "the wait for E buffer i - kEBuf also frees W buffer i - kWBuf");
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
    for (int q = 0; q < kDone; ++q) mbar_init(bar(B_DONE + q), 2);   // CH and CL commits
    for (int q = 0; q < 2; ++q) {
      mbar_init(bar(B_ZFULL + q), kExpWarps);
      mbar_init(bar(B_ZEMPTY + q), 2);   // XR and XI commits
    }
    for (int q = 0; q < kWBuf; ++q) mbar_init(bar(B_WFULL + q), 2);
    for (int q = 0; q < kEBuf; ++q) mbar_init(bar(B_EFULL + q), kExpWarps);
    for (int q = 0; q < kJBuf; ++q) mbar_init(bar(B_JEMPTY + q), kDrainWarps);
    *sAbort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == kXrWarp) {
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
  const int jw = 3 * S.NJ;   // tensor-memory columns of one J buffer (grouped form)
  auto tj_col = [&](int b) { return tbase + (uint32_t)(kWBuf * 2 * S.MP + b * jw); };

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
      // all loads first (n <= 16: at most four variables per warpgroup), so
      // that their latency is paid once
      float2 yv[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int j = wg + 4 * q;
        yv[q] = live && j < n ? y[(size_t)pos * n + j] : make_float2(1.f, 0.f);
      }
      const double tau = live && wg == 0 ? tau_in[pos] : 0.0;
      if (wg == 0)
        ((float*)(zre + P.z_tau))[row] = (float)(tau * (double)S.inv_D * 1.4426950408889634);   // (tau/D) log2(e)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int j = wg + 4 * q;
        if (j >= n) break;
        float rem_r, rem_i;
        log_coords(yv[q], rem_r, rem_i);
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
      // W of unit i full; its issuers waited for the coefficient GEMM of
      // unit i - kEBuf first, so E buffer e is free as well
      if (!wait(B_WFULL + w, use(i, kWBuf))) break;
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
  } else if (warp < kXrWarp) {
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
        float jr[8];
        tmem_ld8_j(tj_col(b) + lane_base + c0, S.NJ, true, jr);
        if (live) {
#pragma unroll
          for (int v = 0; v < 4; ++v) {
            const int u = c0 / 2 + v;
            if (u < n + 2) erow[(size_t)u * 128] = make_float2(jr[2 * v], jr[2 * v + 1]);
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(bar(B_JEMPTY + b));
    }
  } else if (warp < kLoadWarp) {
    // ---------------- MMA issuers: each warp walks its loop together, lane 0
    // issues each MMA and commit.  Four warps on the four SM sub-partitions,
    // each owning its own accumulator columns: XR and XI the Re and Im halves
    // of the exponent GEMM, CH and CL the hi and lo parts of the coefficient
    // GEMM (an MMA holds its issuing thread for about a hundred cycles, so
    // four issuers keep the tensor core four times as busy as one) ----------------
    // a failed (timed-out) wait in any lane stops every lane, so the warp
    // walks the loop together
    auto waitw = [&](int bb, int uu) { return __all_sync(0xffffffffu, wait(bb, uu)); };
    int last = -1;   // the last unit this warp committed
    if (warp == kXrWarp || warp == kXiWarp) {
      const bool im = warp == kXiWarp;
      const uint32_t idx_x = idesc_bf16(128, S.MP), sbo_x = S.KX * 16;
      for (Unit u = first_unit; u.i < U; u = next_unit(u)) {
        const int i = u.i, w = ring(i, kWBuf), c = ring(i, kCBuf), lt = u.lt;
        if (first_of_tile(u) && !waitw(B_ZFULL + (lt & 1), lt >> 1)) break;
        if (!waitw(B_CFULL + c, use(i, kCBuf))) break;
        // E buffer of unit i free: the coefficient GEMM of unit i - kEBuf is
        // done (the exp warps see it through W of unit i, which completes
        // after this wait).  That GEMM was issued after "E full" of unit
        // i - kEBuf = i - kWBuf, which the exp warps signal once they have
        // read its W: so W buffer w is free too, without a wait of its own.
        if (i >= kEBuf && !waitw(B_DONE + ring(i - kEBuf, kDone), use(i - kEBuf, kDone))) break;
        tc_fence_after();
        const uint32_t cb = su32(sm + coff(c));
        const uint32_t za = su32(sm + zoff(lt & 1)) + (im ? (uint32_t)P.z_im : 0u);
        const uint32_t tw = tw_col(w) + (im ? (uint32_t)S.MP : 0u);
        // a K-slice of 256 bytes adds 16 to a descriptor's address field
        const uint64_t bd = smem_desc(cb + S.off_bexp, 128, sbo_x), ad = smem_desc(za, 128, sbo_x);
        for (int s = 0; s < S.KX / 16; ++s) mma_bf16_w(tw, ad + 16 * s, bd + 16 * s, idx_x, s > 0);
        mma_commit_w(bar(B_WFULL + w));
        if (last_of_tile(u)) mma_commit_w(bar(B_ZEMPTY + (lt & 1)));
        last = i;
      }
      if (*sAbort && last >= 0)   // let the MMAs issued land before the CTA's memory goes away
        mbar_wait(bar(B_WFULL + ring(last, kWBuf)), (uint32_t)use(last, kWBuf) & 1u);
    } else {
      const bool lo = warp == kClWarp;
      const uint32_t sbo_c = S.KC * 16;
      for (Unit u = first_unit; u.i < U; u = next_unit(u)) {
        const int i = u.i, e = ring(i, kEBuf), b = ring(i, kJBuf), c = ring(i, kCBuf);
        if (!waitw(B_EFULL + e, use(i, kEBuf))) break;   // E of unit i (and so its constants) ready
        if (i >= kJBuf && !waitw(B_JEMPTY + b, use(i, kJBuf) - 1)) break;
        tc_fence_after();
        const uint32_t cb = su32(sm + coff(c));
        const uint32_t ea = su32(sm + eoff(e)) + (lo ? (uint32_t)P.e_lo : 0u);
        const uint64_t ad = smem_desc(ea, 128, sbo_c), bd = smem_desc(cb + S.off_bhi, 128, sbo_c);
        if (lo)
          coef_gemm_lo(tj_col(b), ad, bd, S.NJ, S.KC / 16);
        else
          coef_gemm_hi(tj_col(b), ad, bd, S.NJ, S.KC / 16);
        mma_commit_w(bar(B_DONE + ring(i, kDone)));
        last = i;
      }
      if (*sAbort && last >= 0)
        mbar_wait(bar(B_DONE + ring(last, kDone)), (uint32_t)use(last, kDone) & 1u);
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
  if (warp == kXrWarp) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(P.tmem_cols));
  }
}

}  // namespace

// Shared memory the pipelined kernel needs for these shapes (0: it does not
// serve them).
int eval_pipe_smem(const MixedSys& s) {
  // the W and J rings in the 512 tensor-memory columns of the SM
  if (s.n > 16 || s.ne != s.n || !s.jst || kWBuf * 2 * s.MP + kJBuf * 3 * s.NJ > 512) return 0;
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
  int cols = kWBuf * 2 * s.MP + kJBuf * 3 * s.NJ, t = 32;
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
