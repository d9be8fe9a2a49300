// Mixed-precision evaluation of the homotopy and its extended Jacobian on the
// fifth-generation tensor cores (tcgen05, accumulators in tensor memory).
//
// Algorithm 2 (Section 5) for tiles of 128 points: a persistent CTA of 256
// threads walks its tiles; point r of a tile is tensor-memory lane r, served
// by thread r of each of the two warpgroups, which split the columns:
//   op. 1   z = log y in FP32 (principal branch) in the units of the
//           exponential, Re z = log2 |y|, Im z = arg y / (2 pi); Re z and
//           Im z each split into three BF16 parts (hi + mid + lo carries the
//           full FP32 value);
//   op. 2a  per equation k: W = Z A_k by tcgen05.mma kind::f16 with FP32
//           accumulation, K = the three splits of the n coordinates; the
//           integer exponents are exact in BF16.  Re W and Im W are two MMAs
//           that share the B operand;
//   exp     E = 2^(Re W + (tau/D) log2(e) e) (cos 2 pi r, sin 2 pi r),
//           r = Im W - rint(Im W): the t-exponent term is added in FP32 (e
//           exact in FP32), the phase in revolutions is reduced modulo 1 by one
//           exact subtraction before the MUFU sine/cosine; E is split into
//           BF16 hi + lo and written as the A operand of op. 2b (cexp_split8,
//           shared with the pipelined step kernel);
//   op. 2b  [D_z h_k | D_tau h_k | h_k] = E_k B_k^T as a real GEMM on
//           [Re E, Im E] x [[Re B, Im B], [-Im B, Re B]]^T, three passes
//           hi*hi + hi*lo + lo*hi, FP32 accumulation in tensor memory;
//   op. 3   D_y h_k = D_z h_k diag(1/y) for the caller's H_y.  The step's
//           scratch keeps D_z h_k instead: the solve applies diag(1/y) to
//           its two n-vector solutions (n products per path, not n^2).
// The per-equation constants (exponent operand and e, then B_k hi/lo) are one
// contiguous image per equation, double-buffered into shared memory with
// cp.async.bulk (the bulk-copy engine) while the previous equation computes;
// large shapes prefetch only the exponent part (see launch_core).
// Operands use the canonical K-major layout without swizzle (8 x 16-byte core
// matrices; K-adjacent cores 128 bytes apart, 8-row groups K*16 bytes apart).
// Every wait on an mbarrier is bounded (about two seconds of global time);
// a wait that gives up sets the device error flag and the CTA winds down.
#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>

#include "hpt_internal.h"
#include "hpt_tc.cuh"

namespace hpt {
namespace {

struct MixedArgs {
  MixedSys sys;   // the system of a single-system launch
  int tmem_cols;
  int nbuf;   // constant-image buffers: 2 (prefetch next equation) or 1
  int split;  // 1: the buffers hold only the exponent part; the coefficient part
              // has one buffer of its own (s_cpart), refilled once its GEMM is done
  int wbuf;   // exponent accumulators W in tensor memory: 2 (next GEMM under the epilogue) or 1
  // shared-memory carve-up (bytes from the 1024-aligned base)
  int s_are, s_aim, s_invy, s_achi, s_aclo, s_const0, s_const1, s_cpart, s_bar;
  int s_zq;   // fixed angles of the tile's points ([j][128] uint32) when a system has large exponents
  int64_t p;
  int ntiles;
};

constexpr int kEvalThreads = 256;   // two warpgroups over the 128 TMEM lanes

// Barriers in shared memory: [0], [1] constant buffers; [2], [3] exponent
// accumulators W[0], W[1]; [4] coefficient accumulator J; [5] coefficient
// part buffer (split mode).
// MAP: positions come from a position map (many systems); otherwise position
// = path of the single system described by P.sys.
// SPLIT: the constant buffers hold only the exponent parts; the coefficient
// part has a buffer of its own (large shapes; a compile-time choice, so that
// the other form carries none of its code).
template <bool MAP, bool SPLIT>
__global__ void __launch_bounds__(kEvalThreads, 2)
eval_mixed_kernel(MixedArgs P, const float2* __restrict__ y, const double* __restrict__ tin, int tau_is_t,
                  const uint8_t* __restrict__ chunks, float2* __restrict__ ext, float2* __restrict__ oH,
                  float2* __restrict__ oHy, float2* __restrict__ oHt, int32_t* __restrict__ err, PathMap pm_in) {
  const PathMap pm = MAP ? pm_in : PathMap();   // null pointers fold away in the single-system form
  extern __shared__ uint8_t smem_raw[];
  uint8_t* sm = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* sAre = sm + P.s_are;
  uint8_t* sAim = sm + P.s_aim;
  float2* sInvY = (float2*)(sm + P.s_invy);        // [n][128]
  uint8_t* sAcHi = sm + P.s_achi;
  uint8_t* sAcLo = sm + P.s_aclo;
  uint64_t* bars = (uint64_t*)(sm + P.s_bar);
  uint32_t* tslot = (uint32_t*)(sm + P.s_bar + 64);
  int* sAbort = (int*)(sm + P.s_bar + 68);

  const int tid = threadIdx.x, warp = tid >> 5;
  const int row = tid & 127;          // point of the tile = TMEM lane
  const int half = tid >> 7;          // warpgroup: splits the column chunks
  const int ntiles = pm.npos ? (*pm.npos + 127) / 128 : P.ntiles;
  // A CTA's work items are (tile, range of equations) pairs; the evaluation
  // of one (tile, equation) is the same whichever CTA does it.  Many
  // systems: whole tiles, strided over the grid.  One system: the sequence
  // of (tile, equation) units, tile-major, is cut into gridDim.x contiguous
  // ranges of equal length (to within one unit), so every CTA does the same
  // work whether the tiles outnumber the CTAs or not; a range that crosses
  // tile boundaries is one item per tile it touches.
  const int64_t units = MAP ? 0 : (int64_t)ntiles * P.sys.ne;
  const int64_t u0 = (int64_t)blockIdx.x * units / (int64_t)gridDim.x;
  const int64_t u1 = ((int64_t)blockIdx.x + 1) * units / (int64_t)gridDim.x;
  const int t0 = MAP ? 0 : (int)(u0 / P.sys.ne);
  const int my_tiles = MAP ? (ntiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x
                           : (u1 > u0 ? (int)((u1 - 1) / P.sys.ne) - t0 + 1 : 0);
  if (my_tiles <= 0) return;
  const bool lookahead = P.nbuf == 2 && P.wbuf == 2;
  const int nmax = pm.nmax ? pm.nmax : P.sys.n;
  auto tile_of = [&](int it) { return MAP ? (int)blockIdx.x + it * (int)gridDim.x : t0 + it; };
  auto sys_of = [&](int tile) { return pm.tile_sys ? pm.tile_sys[tile] : 0; };
  // equations [kb, ke) of work item it (ln: the tile's equation count)
  auto krange = [&](int it, int ln, int& kb, int& ke) {
    if (MAP) {
      kb = 0;
      ke = ln;
      return;
    }
    const int64_t base = (int64_t)tile_of(it) * ln;
    kb = (int)(u0 > base ? u0 - base : 0);
    ke = (int)(u1 - base < (int64_t)ln ? u1 - base : (int64_t)ln);
  };

  if (tid == 0) {
    // 2, 3 (W full) and 4 (J full): warps 0 and 1 commit
    for (int i = 0; i < (SPLIT ? 6 : 5); ++i) mbar_init(su32(&bars[i]), i >= 2 && i <= 4 ? 2 : 1);
    *sAbort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tslot)),
                 "r"(P.tmem_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = *tslot;
  const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;

  auto cbuf = [&](int g) -> uint8_t* { return sm + ((P.nbuf == 2 && (g & 1)) ? P.s_const1 : P.s_const0); };
  auto cpar = [&](int g) -> uint32_t { return (uint32_t)(P.nbuf == 2 ? (g >> 1) : g) & 1u; };

  // exponent GEMM of work item g (an equation of system S) into W[g & 1];
  // the whole of warps 0 and 1, the Re and the Im half (lane 0 issues; the
  // operands stay warp-uniform)
  auto issue_exp = [&](int g, const MixedSys& S) -> bool {
    if (!__all_sync(0xffffffffu, mbar_wait(su32(&bars[P.nbuf == 2 ? (g & 1) : 0]), cpar(g)))) return false;
    tc_fence_after();
    const uint32_t cb = su32(cbuf(g));
    const uint32_t tw = tbase + (uint32_t)((P.wbuf == 2 ? (g & 1) : 0) * 2 * S.MP);
    const uint32_t idx_x = idesc_bf16(128, S.MP), sbo_x = S.KX * 16;
    // a K-slice of 256 bytes adds 16 to a descriptor's address field
    const uint64_t bd = smem_desc(cb + S.off_bexp, 128, sbo_x);
    const bool im = warp == 1;
    const uint64_t ad = smem_desc(su32(im ? sAim : sAre), 128, sbo_x);
    const uint32_t td = tw + (im ? (uint32_t)S.MP : 0u);
    for (int s = 0; s < S.KX / 16; ++s) mma_bf16_w(td, ad + 16 * s, bd + 16 * s, idx_x, s > 0);
    mma_commit_w(su32(&bars[2 + (g & 1)]));
    return true;
  };

  // constant images for the first nbuf work items; (lit, lk) is the next
  // item to load, `issued` the number of items loaded so far (thread 0).  In
  // split mode these loads carry the exponent part only and a second cursor
  // (cit, ck, cissued) loads the coefficient parts, one item ahead.
  int lit = 0, lk = 0, issued = 0;
  int cit = 0, ck = 0, cissued = 0;
  {
    int kb0, ke0;
    krange(0, pm.sys_tab ? pm.sys_tab[sys_of(tile_of(0))].ne : P.sys.ne, kb0, ke0);
    lk = ck = kb0;
  }
  auto load_item = [&](int& xit, int& xk, bool cpart) {
    const int ls = sys_of(tile_of(xit));
    const int ln = pm.sys_tab ? pm.sys_tab[ls].ne : P.sys.ne;   // one image per equation
    const int lbytes = pm.sys_tab ? pm.sys_tab[ls].chunk_bytes : P.sys.chunk_bytes;
    const int lsplit = pm.sys_tab ? pm.sys_tab[ls].off_bhi : P.sys.off_bhi;
    const int64_t loff = pm.sys_tab ? pm.sys_tab[ls].chunk_off : P.sys.chunk_off;
    const uint8_t* src = chunks + loff + (size_t)xk * lbytes;
    if (cpart) {
      bulk_load(su32(sm + P.s_cpart), src + lsplit, lbytes - lsplit, su32(&bars[5]));
    } else {
      bulk_load(su32(cbuf(issued)), src, SPLIT ? lsplit : lbytes, su32(&bars[P.nbuf == 2 ? (issued & 1) : 0]));
    }
    int kb, ke;
    krange(xit, ln, kb, ke);
    if (++xk >= ke) {
      ++xit;
      if (xit < my_tiles) {
        const int nl = pm.sys_tab ? pm.sys_tab[sys_of(tile_of(xit))].ne : P.sys.ne;
        krange(xit, nl, kb, ke);
        xk = kb;
      }
    }
  };
  auto load_next = [&]() {
    if (lit >= my_tiles) return;
    load_item(lit, lk, false);
    ++issued;
  };
  auto load_cnext = [&]() {
    if (!SPLIT || cit >= my_tiles) return;
    load_item(cit, ck, true);
    ++cissued;
  };
  if (tid == 0) {
    for (int q = 0; q < P.nbuf; ++q) load_next();
    load_cnext();
  }
  int g = 0;

  for (int it = 0; it < my_tiles; ++it) {
    const int tile = tile_of(it);
    const MixedSys S = pm.sys_tab ? pm.sys_tab[sys_of(tile)] : P.sys;
    const int n = S.n, ne = S.ne;   // variables, equations
    int kb, ke;
    krange(it, ne, kb, ke);
    const uint32_t t_j = tbase + (uint32_t)(P.wbuf * 2 * S.MP);
    const int64_t pos = (int64_t)tile * 128 + row;   // position of this row
    const int64_t path = pm.list ? pm.list[pos] : pos;
    const bool live = pm.list ? path >= 0 : pos < P.p;
    const size_t vbase = !live ? 0 : (pm.vofs ? (size_t)pm.vofs[path] : (size_t)path * n);
    const float inv_D = S.inv_D;
    // ---- op. 1: z = log y, three-way BF16 split, 1/y (variables split by half)
    const double tv = (live && tin) ? tin[path] : (tau_is_t ? 1.0 : 0.0);
    const double tau = tau_is_t ? log(tv) : tv;
    const float tau2 = (float)(tau * (double)inv_D * 1.4426950408889634);   // (tau / D) log2(e)
    const float t_inv = (float)(tau_is_t ? 1.0 / tv : exp(-tau));
    uint32_t* sZq = (uint32_t*)(sm + P.s_zq);
    for (int j = half; j < n; j += 2) {
      float2 v = live ? y[vbase + j] : make_float2(1.f, 0.f);
      float zr, zi;
      log_coords(v, zr, zi);
      if (S.off_aint) sZq[j * 128 + row] = fixed_angle(zi);
      if (oHy) {
        const float r2 = v.x * v.x + v.y * v.y;
        sInvY[j * 128 + row] = make_float2(v.x / r2, -v.y / r2);
      }
      float rem_r = zr, rem_i = zi;
#pragma unroll
      for (int s = 0; s < 3; ++s) {
        const uint16_t hr = bf16_rn(rem_r), hi = bf16_rn(rem_i);
        *(uint16_t*)(sAre + canon(row, s * n + j, S.KX)) = hr;
        *(uint16_t*)(sAim + canon(row, s * n + j, S.KX)) = hi;
        rem_r -= bf16_f(hr);
        rem_i -= bf16_f(hi);
      }
    }
    for (int q = 3 * n + half; q < S.KX; q += 2) {
      *(uint16_t*)(sAre + canon(row, q, S.KX)) = 0;
      *(uint16_t*)(sAim + canon(row, q, S.KX)) = 0;
    }
    proxy_fence();
    tc_fence_before();
    __syncthreads();
    if (warp < 2 && lookahead && !issue_exp(g, S)) atomicExch(sAbort, 1);

    // row kk of the outputs from J: 8-column chunks (4 complex entries)
    // alternate between the warpgroups (NJ is a multiple of 16)
    auto write_row = [&](int kk) {
      const uint32_t tj = t_j + lane_base;
      // the step scratch row [D_z h_kk | D_tau h_kk | h_kk] is contiguous in u
      // with stride 128 (ext_index); the solve applies diag(1/y)
      float2* erow = ext ? ext + ext_index(pos, kk, 0, nmax) : nullptr;
      for (int c0 = 8 * half; c0 < S.NJ; c0 += 16) {
        float jr[8];
        tmem_ld8_j(tj + c0, S.NJ, S.jst != 0, jr);
        if (!live) continue;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int u = c0 / 2 + q;
          const float2 v = make_float2(jr[2 * q], jr[2 * q + 1]);
          if (erow) {
            if (u < n + 2) erow[(size_t)u * 128] = v;
            continue;
          }
          if (u < n) {
            if (oHy) {
              const float2 iy = sInvY[u * 128 + row];
              oHy[((size_t)path * ne + kk) * n + u] = make_float2(v.x * iy.x - v.y * iy.y, v.x * iy.y + v.y * iy.x);
            }
          } else if (u == n) {
            if (oHt) oHt[(size_t)path * ne + kk] = make_float2(v.x * t_inv, v.y * t_inv);
          } else if (u == n + 1) {
            if (oH) oH[(size_t)path * ne + kk] = v;
          }
        }
      }
    };

    for (int k = kb; k < ke; ++k, ++g) {
      // ---- op. 2a: W = Z A_k (exponent GEMM); with two constant buffers the
      // GEMM of equation k+1 is issued now and runs under this epilogue
      if (warp < 2) {
        const bool ok1 = lookahead ? (k + 1 < ke ? issue_exp(g + 1, S) : true) : issue_exp(g, S);
        if (!ok1) atomicExch(sAbort, 1);
      }
      bool ok = mbar_wait(su32(&bars[P.nbuf == 2 ? (g & 1) : 0]), cpar(g));   // e of equation k visible
      ok = __all_sync(0xffffffffu, ok && mbar_wait(su32(&bars[2 + (g & 1)]), (uint32_t)(g >> 1) & 1u));
      if (!ok) atomicExch(sAbort, 1);
      tc_fence_after();
      // ---- complex exponential, BF16 hi/lo split into the op. 2b A operand
      {
        const float* texp = (const float*)(cbuf(g) + S.off_texp);
        const uint32_t tw = tbase + (uint32_t)((P.wbuf == 2 ? (g & 1) : 0) * 2 * S.MP) + lane_base;
        // chunks of 8 monomials alternate between the warpgroups (MP is a
        // multiple of 16, so both get the same number)
        for (int c0 = 8 * half; c0 < S.MP; c0 += 16) {
          uint32_t wre[8], wim[8];
          tmem_ld8(tw + c0, wre);
          tmem_ld8(tw + S.MP + c0, wim);
          tmem_wait_ld();
          uint4 hre, lre, him, lim;
          const uint32_t big8 =
              S.off_bigm ? (((const uint32_t*)(cbuf(g) + S.off_bigm))[c0 >> 5] >> (c0 & 31)) & 0xffu : 0u;
          cexp_split8(wre, wim, texp + c0, tau2, big8, (const int16_t*)(cbuf(g) + S.off_aint) + c0 * n,
                      sZq + row, n, hre, lre, him, lim);
          // Re E at K = c0.., Im E at K = MP + c0..; 8 values = one core column
          *(uint4*)(sAcHi + canon(row, c0, S.KC)) = hre;
          *(uint4*)(sAcLo + canon(row, c0, S.KC)) = lre;
          *(uint4*)(sAcHi + canon(row, S.MP + c0, S.KC)) = him;
          *(uint4*)(sAcLo + canon(row, S.MP + c0, S.KC)) = lim;
        }
      }
      proxy_fence();
      tc_fence_before();
      __syncthreads();
      if (*sAbort) goto teardown;
      // ---- op. 2b: [D_z h | D_tau h | h] = E_k B_k^T, split passes.  Lane 0
      // of warp 0 issues (operands warp-uniform); in the grouped form warp 1
      // issues the E_lo part at the same time (an MMA holds its issuing
      // thread for about a hundred cycles).  Both commit.
      if (warp < 2) {
        // split mode: the coefficient part of item g in its own buffer
        if (SPLIT && !__all_sync(0xffffffffu, mbar_wait(su32(&bars[5]), (uint32_t)g & 1u))) atomicExch(sAbort, 1);
        tc_fence_after();
        // cb + off_bhi addresses the coefficient part in either layout
        const uint32_t cb = SPLIT ? su32(sm + P.s_cpart) - (uint32_t)S.off_bhi : su32(cbuf(g));
        const uint32_t sbo_c = S.KC * 16;
        const uint64_t ahd = smem_desc(su32(sAcHi), 128, sbo_c), ald = smem_desc(su32(sAcLo), 128, sbo_c);
        const uint64_t bhd = smem_desc(cb + S.off_bhi, 128, sbo_c);
        if (S.jst) {
          if (warp == 0)
            coef_gemm_hi(t_j, ahd, bhd, S.NJ, S.KC / 16);
          else
            coef_gemm_lo(t_j, ald, bhd, S.NJ, S.KC / 16);
        } else if (warp == 0) {
          coef_gemm(t_j, ahd, ald, bhd, smem_desc(cb + S.off_blo, 128, sbo_c), S.NJ, S.KC / 16, false);
        }
        mma_commit_w(su32(&bars[4]));   // warp 1 without MMAs: arrives at once
      }
      ok = __all_sync(0xffffffffu, mbar_wait(su32(&bars[4]), (uint32_t)g & 1u));
      if (!ok) atomicExch(sAbort, 1);
      tc_fence_after();
      // both GEMMs of equation k are done: its constant buffer and the E
      // operand are free
      if (tid == 0 && ok) {
        proxy_fence();
        load_next();    // item g + nbuf into this buffer
        load_cnext();   // split mode: coefficient part of item g + 1
      }
      if (ok) write_row(k);
      tc_fence_before();
      __syncthreads();
      if (*sAbort) goto teardown;
    }
  }

teardown:
  if (*sAbort) {
    if (tid == 0) {
      atomicExch(err, 1);
      // let copies and MMAs still in flight land before the CTA's resources go away
      for (int q = g; q < issued; ++q) mbar_wait(su32(&bars[P.nbuf == 2 ? (q & 1) : 0]), cpar(q));
      if (SPLIT)
        for (int q = g; q < cissued; ++q) mbar_wait(su32(&bars[5]), (uint32_t)q & 1u);
      mbar_wait(su32(&bars[2 + (g & 1)]), (uint32_t)(g >> 1) & 1u);
      mbar_wait(su32(&bars[2 + ((g + 1) & 1)]), (uint32_t)((g + 1) >> 1) & 1u);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(P.tmem_cols));
  }
}

// One CTA waits on an mbarrier that nothing completes, with the bounded wait
// of the evaluation kernel: it gives up after ~2 s and raises the error flag
// (the failure path, exercised without a device fault).
__global__ void bounded_wait_probe_kernel(int32_t* __restrict__ err) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(su32(&bar), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const bool ok = mbar_wait(su32(&bar), 0);   // no arrival: times out
  if (!ok && threadIdx.x == 0) atomicExch(err, 1);
}

int g_num_sms = 0;

int num_sms() {
  if (!g_num_sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_num_sms <= 0) g_num_sms = 1;
  }
  return g_num_sms;
}

// Shared-memory carve-up for the largest shapes of a launch (maxs), the
// single-system arguments (sys) and the grid; then the launch.
cudaError_t launch_core(hpt_system prof, const MixedSys& sys, const MixedSys& maxs, int64_t p, int64_t ntiles,
                        const uint8_t* chunks, const void* y, const double* tin, int tau_is_t, const EvalOut& out,
                        int32_t* err, const PathMap& pm, int ctas_per_sm, cudaStream_t st) {
  if (ntiles > 0x7fffffff) return cudaErrorInvalidValue;
  const bool map = pm.list != nullptr;
  auto pick = [map](bool split) {
    return map ? (split ? eval_mixed_kernel<true, true> : eval_mixed_kernel<true, false>)
               : (split ? eval_mixed_kernel<false, true> : eval_mixed_kernel<false, false>);
  };
  int dev = 0, max_smem = 0, sm_smem = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaDeviceGetAttribute(&sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  // Configurations in order of preference, the first that fits wins:
  // (nbuf, wbuf, split) = (2, 2, 0) prefetches the next equation's constants
  // and issues its exponent GEMM into the second W accumulator under the
  // current epilogue; (2, 2, 1) prefetches only the exponent parts and loads
  // each coefficient part once the previous coefficient GEMM is done (in time
  // for its own GEMM after the epilogue: large shapes); (1, 2, 0) has no
  // prefetch; (1, 1, 0) needs the least shared and tensor memory (it is the
  // one that serves m_k up to 128).  At n = 16 the overlap is worth more than residency:
  // (1, 1) with three CTAs per SM measured 177 us against 117 us for (2, 2)
  // with two.  Residency is bounded by shared memory, registers and the 512
  // tensor-memory columns of an SM; a persistent grid above it would run in
  // two waves.
  MixedArgs best{};
  int best_smem = 0, best_per_sm = 0;
  cudaError_t e = cudaSuccess;
  const int cfg[4][3] = {{2, 2, 0}, {2, 2, 1}, {1, 2, 0}, {1, 1, 0}};
  auto r128 = [](int v) { return (v + 127) / 128 * 128; };
  const int xpart = r128(std::max(maxs.off_bhi, maxs.MP * maxs.KX * 2 + maxs.MP * 4));   // largest exponent part
  const int cpart = r128(2 * maxs.NJ * maxs.KC * 2);             // largest coefficient part
  for (const auto& c : cfg) {
    MixedArgs a;
    a.sys = sys;
    a.nbuf = c[0];
    a.wbuf = c[1];
    a.split = c[2];
    int cols = a.wbuf == 2 ? maxs.tcols2 : maxs.tcols1, t = 32;   // W buffers, coefficient accumulator
    while (t < cols) t *= 2;
    if (t > 512) continue;
    a.tmem_cols = t;
    int off = 0;
    auto take = [&](int bytes) {
      int o = off;
      off += (bytes + 1023) / 1024 * 1024;
      return o;
    };
    a.s_are = take(128 * maxs.KX * 2);
    a.s_aim = take(128 * maxs.KX * 2);
    a.s_invy = take(out.Hy ? 128 * maxs.n * 8 : 0);   // 1/y only for the caller's H_y
    a.s_zq = take(maxs.off_aint ? 128 * maxs.n * 4 : 0);
    a.s_achi = take(128 * maxs.KC * 2);
    a.s_aclo = take(128 * maxs.KC * 2);
    const int cbytes = a.split ? xpart : maxs.chunk_bytes;
    a.s_const0 = take(cbytes);
    a.s_const1 = a.nbuf == 2 ? take(cbytes) : a.s_const0;
    a.s_cpart = a.split ? take(cpart) : a.s_const0;
    a.s_bar = take(128);
    a.p = p;
    a.ntiles = (int)ntiles;
    const int smem = off + 1024;   // slack for aligning the dynamic base
    if (smem > max_smem) continue;
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, pick(a.split));
    if (e != cudaSuccess) return e;
    const int regs_per_cta = (fa.numRegs + 7) / 8 * 8 * kEvalThreads;
    // 1 KB of shared memory per CTA is reserved by the system
    const int per_sm = std::min({sm_smem / (smem + 1024), 65536 / regs_per_cta, 512 / a.tmem_cols});
    if (per_sm >= 1) {
      best = a;
      best_smem = smem;
      best_per_sm = per_sm;
      break;
    }
  }
  if (best_per_sm < 1) return cudaErrorInvalidConfiguration;
  auto kern = pick(best.split);
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, best_smem);
  if (e != cudaSuccess) return e;
  const int per_sm = ctas_per_sm > 0 ? std::min(ctas_per_sm, best_per_sm) : best_per_sm;
  const int64_t slots = (int64_t)num_sms() * per_sm;
  // One system: the (tile, equation) units are shared out in equal
  // contiguous ranges (see the kernel), so with few tiles a tile's equations
  // go to several CTAs and with many the last wave is not left to part of
  // the SMs (512 tiles on 304 slots: 27 units per CTA instead of 2 tiles
  // on some CTAs and 1 on others).  The grid is the fewest CTAs that still
  // give the smallest range length.
  int64_t grid = slots;
  if (!map) {
    const int64_t units = ntiles * sys.ne;
    const int64_t per = (units + slots - 1) / slots;
    grid = per > 0 ? (units + per - 1) / per : 0;
  } else if (grid > ntiles) {
    grid = ntiles;
  }
  if (grid < 1) return cudaSuccess;
  int pi = prof_begin(prof, "eval_mixed_tc", st);
  kern<<<(unsigned)grid, kEvalThreads, best_smem, st>>>(best, (const float2*)y, tin, tau_is_t, chunks,
                                                       (float2*)out.ext, (float2*)out.H, (float2*)out.Hy,
                                                       (float2*)out.Ht, err, pm);
  prof_end(prof, pi, st);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_bounded_wait_probe(int32_t* err, cudaStream_t st) {
  bounded_wait_probe_kernel<<<1, 32, 0, st>>>(err);
  return cudaGetLastError();
}

bool eval_mixed_fits(int n, int MP, int KX, int NJ, int KC, int chunk_bytes, bool big, bool grouped, int max_smem) {
  auto r = [](int v) { return (v + 1023) / 1024 * 1024; };
  // the leanest configuration (one constant buffer, one W accumulator), 1/y
  // and the fixed angles of large exponents included
  const int smem = r(128 * KX * 2) * 2 + r(128 * n * 8) + (big ? r(128 * n * 4) : 0) + r(128 * KC * 2) * 2 +
                   r(chunk_bytes) + r(128) + 1024;
  return smem <= max_smem && 2 * MP + (grouped ? 3 : 1) * NJ <= 512;
}

int eval_mixed_max_ctas(int tmem_cols) { return 512 / tmem_cols >= 2 ? 2 : 1; }

MixedSys mixed_sys_of(const hpt_system s) {
  const MixedLayout& L = s->ml;
  MixedSys m;
  m.n = s->nv;
  m.ne = s->n;
  m.MP = L.MP;
  m.KX = L.KX;
  m.NJ = L.NJ;
  m.KC = L.KC;
  m.chunk_bytes = L.chunk_bytes;
  m.off_bexp = L.off_bexp;
  m.off_bhi = L.off_bhi;
  m.off_blo = L.off_blo;
  m.off_texp = L.off_texp;
  m.jst = L.grouped ? 1 : 0;
  m.tcols1 = 2 * L.MP + (m.jst ? 3 : 1) * L.NJ;
  m.tcols2 = 4 * L.MP + (m.jst ? 3 : 1) * L.NJ;
  m.off_bigm = L.off_bigm;
  m.off_aint = L.off_aint;
  m.inv_D = (float)(1.0 / (double)s->D);
  m.chunk_off = 0;
  return m;
}

cudaError_t launch_eval_mixed(hpt_system s, int64_t p, const void* y, const double* tin, int tau_is_t,
                              const EvalOut& out, cudaStream_t st) {
  if (p <= 0) return cudaSuccess;
  const MixedSys m = mixed_sys_of(s);
  // the step's evaluation (the scratch only, tau given): the pipelined kernel
  // where its shapes fit (same arithmetic, same bits)
  if (out.ext && !out.H && !out.Hy && !out.Ht && !tau_is_t && tin) {
    const int need = eval_pipe_smem(m);
    int dev = 0, max_smem = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (need > 0 && need <= max_smem)
      return launch_eval_pipe(s, m, p, s->d_chunks, y, tin, out.ext, s->d_err, num_sms(), st);
  }
  return launch_core(s, m, m, p, (p + 127) / 128, s->d_chunks, y, tin, tau_is_t, out, s->d_err, PathMap(), 0,
                     st);
}

cudaError_t launch_eval_mixed_map(hpt_system prof, const MixedSys& maxs, int tmem_cols, const uint8_t* chunks,
                                  int64_t p, const void* y, const double* tau, const PathMap& pm, void* ext,
                                  int32_t* err, int ctas_per_sm, cudaStream_t st) {
  if (p <= 0) return cudaSuccess;
  if (!pm.list || !pm.tile_sys || !pm.vofs || !pm.npos || !pm.sys_tab || maxs.n != pm.nmax)
    return cudaErrorInvalidValue;
  EvalOut out;
  out.ext = ext;
  (void)tmem_cols;
  return launch_core(prof, maxs, maxs, p, (p + 127) / 128, chunks, y, tau, 0, out, err, pm, ctas_per_sm, st);
}

}  // namespace hpt
