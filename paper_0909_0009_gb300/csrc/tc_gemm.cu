// Legendre transforms of the mixed-precision forms on the 5th-generation tensor cores.
//
// Both transforms are batched GEMMs over the problems (m, parity) with the 2 N_r real
// columns c of all shells as the M dimension (one or two 128-row tiles):
//   synthesis (step (ii)):  F[mp][j][c]  = sum_k  Phi[mp][k][c] * Lambda_syn[mp][j][k]
//                           M = c, N = ring pairs j, K = degrees k
//   analysis  (step (iv)):  Phi[mp][k][c] = sum_j G[mp][j][c] * Lambda_ana[mp][k][j]
//                           M = c, N = degrees k, K = ring pairs j
// A (data: Phi or G) is stored with c contiguous and is read MN-major; B (the Legendre
// tables) is stored K-contiguous.  Operands are split into BF16 terms x = x0 + x1 (+ x2)
// and every product of terms whose indices sum to less than the term count is
// accumulated in FP32 in tensor memory (3 products for 2 terms, 6 for 3 terms).
//
// Kernel structure (one persistent CTA per SM, 448 threads; the producer and MMA loops run on
// one lane each, with no warp-wide exchange per stage):
//   warp 0      TMA producer, stages 64 deep in k: one box of A (per term 128 c x 64 k: both
//               64-column halves through a view with a dimension over the halves, 128B
//               swizzle) and one of B (per term nmax rows x two 32-deep slabs, 64B swizzle),
//               each carrying every BF16 term through a last dimension over the terms: two
//               boxes per stage of 28-32 KB each (4 KB boxes move about a sixth of what 32 KB
//               boxes do per clock)
//   warp 1      allocates 512 TMEM columns and issues tcgen05.mma (M = 128, N = tile width
//               up to 256, K = 16) from one thread, up to 4 k steps per stage and one commit
//               per stage (each commit costs the pipe a few hundred cycles); the descriptors of
//               every term and k step are constant offsets from one base per stage.  The leading product and the
//               correction products accumulate in two TMEM accumulators (`cols` apart); the
//               accumulator sets that fit (1 for 256-wide tiles, 2 for 128) rotate over tiles
//   warps 2-13  epilogue, three warps per TMEM lane quadrant taking turns over the tile's
//               column chunks (16 columns for the synthesis and the quadrature, 32 for the
//               per-shell coefficients; more warps keep more F stores in flight): tcgen05.ld
//               of the accumulator, then per mode:
//               synthesis -> F (FP32); analysis -> radial quadrature of Eq. 5 reduced over
//               the shells of the tile (T and E), or the per-shell coefficients.
// Every mbarrier wait is bounded; on expiry the kernel records an error code and unwinds.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <vector>

#include "fnl_internal.cuh"
#include "tc_gemm.cuh"
#include "tc_ptx.cuh"

namespace fnl {

namespace {

// Tensor maps of the instances of a multi-instance launch (see TcArgs::multi).
__constant__ CUtensorMap c_tc_maps[kTcMaxInst * 3];

constexpr int kEpiWarps = 12;                // per TMEM lane quadrant kEpiPerQuad warps take turns
constexpr int kEpiPerQuad = kEpiWarps / 4;  // over a tile's column chunks
constexpr int kThreadsTc = 64 + 32 * kEpiWarps;

// Instruction descriptor, kind::f16: BF16 x BF16 -> FP32, A MN-major, B K-major, M = 128.
__device__ __forceinline__ uint32_t idesc_bf16(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | ((uint32_t)(n >> 3) << 17) | ((128u >> 4) << 24);
}

// Bounded rendezvous of the epilogue warps on an mbarrier (count = kEpiWarps): one arrive
// per warp, then every lane waits for the phase.  Returns false if the wait expired.
__device__ __forceinline__ bool epi_sync(uint64_t* bar, uint32_t parity, int lane, int* err) {
  __syncwarp();
  if (lane == 0) mbar_arrive(bar);
  const bool ok = mbar_wait(bar, parity, err, 5);
  __syncwarp();
  return ok;
}

// The MMAs of one stage: nh (1 or 2) slabs of 32 k, each two k steps of 16, every product of
// terms (ta, tb) with ta + tb < NT.  da, db: descriptors of term 0 of A and B in this stage;
// the other terms and k steps are constant offsets (descriptor start addresses count 16-byte
// units): A k step kk starts 16 rows (2048 B) further, B slab h sits nmax * 64 B after slab 0
// and its second k step 32 B into the swizzled rows.  With SPLIT the leading product
// accumulates in d and the corrections in dc.
template <int NT, bool SPLIT>
__device__ __forceinline__ void issue_stage(uint64_t da, uint64_t db, uint32_t bterm16, uint32_t bslab16, int nh,
                                            uint32_t d, uint32_t dc, uint32_t idesc, bool first) {
#pragma unroll
  for (int kk = 0; kk < 4; ++kk) {
    if (kk >= 2 * nh) break;
    int corr = 0;
#pragma unroll
    for (int ta = 0; ta < NT; ++ta) {
#pragma unroll
      for (int tb = 0; ta + tb < NT; ++tb) {
        const uint64_t ad = da + (uint64_t)((ta * kTcABytes + kk * 2048u) >> 4);
        const uint64_t bd = db + (uint64_t)(tb * bterm16 + (kk >> 1) * bslab16 + (((kk & 1) * 32) >> 4));
        if (SPLIT && (ta | tb)) {
          tc_mma(dc, ad, bd, idesc, (first && kk == 0 && corr == 0) ? 0u : 1u);
          ++corr;
        } else {
          tc_mma(d, ad, bd, idesc, (first && kk == 0 && ta == 0 && tb == 0) ? 0u : 1u);
        }
      }
    }
  }
}

// MODE (TcMode) is a template parameter, so that each mode's kernel is compiled with only its own
// epilogue (the quadrature's registers do not weigh on the synthesis, and the other way round).
template <bool MULTI, int MODE>
__global__ void __launch_bounds__(kThreadsTc, 1) k_tc_gemm(const __grid_constant__ TcArgs a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int S = a.stages;
  const uint32_t bBytes = (uint32_t)a.nmax * 64u * kTcSlabs;  // B bytes per term and stage
  const uint32_t stageBytes = (uint32_t)a.nterms * (kTcABytes + bBytes);
  uint64_t* full = (uint64_t*)(smem + (size_t)S * stageBytes);
  uint64_t* empty = full + S;
  uint64_t* tfull = empty + S;
  uint64_t* tempty = tfull + 2;
  uint64_t* drain = tempty + 2;
  uint64_t* epib = drain + 1;  // [2] rendezvous of the epilogue warps
  uint32_t* tslot = (uint32_t*)(epib + 2);
  // analysis: [4 quadrants][nmax degree columns][2 fields][2 parts][hi, lo] double-float partials of
  // the quadrature, then [kEpiWarps][256] scratch of the epilogue warps
  float* red = (float*)(smem + (size_t)S * stageBytes + 1024);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t sbase = smem_u32(smem);

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&tfull[i], 1);
      mbar_init(&tempty[i], kEpiWarps);
    }
    mbar_init(drain, 1);
    mbar_init(&epib[0], kEpiWarps);
    mbar_init(&epib[1], kEpiWarps);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(tslot))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  if (warp == 0) {
    // ------------------------------------------------------------------ TMA producer
    // Lane 0 alone walks the loop, waits and issues (no warp-wide exchange per stage).
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      uint32_t armed = 0, armed_par = 0;  // stages with copies issued, and the parity armed
      int prev_inst = -1;
      for (int t = blockIdx.x; t < a.ntiles && ok; t += gridDim.x) {
        const TcTile tl = a.tiles[t];
        const CUtensorMap* mA = MULTI ? c_tc_maps + 3 * tl.inst : &a.one.tmA;
        const CUtensorMap* mB = MULTI ? c_tc_maps + 3 * tl.inst + 1 : &a.one.tmB;
        if (MULTI && tl.inst != prev_inst) {
          // bring this instance's tensor maps into the copy engine's descriptor cache
          asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)mA) : "memory");
          asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)mB) : "memory");
        }
        prev_inst = tl.inst;
        const int nst = (tl.nkb + kTcSlabs - 1) / kTcSlabs;
        for (int sg = tl.kb0 / kTcSlabs; sg < nst; ++sg) {
          if (!mbar_wait_fast(&empty[stage], phase ^ 1, a.err, 1)) {
            ok = false;
            break;
          }
          // boxes past the end of a tensor are zero-filled; a second slab past the tile's
          // last k block is loaded but never read by the MMAs
          mbar_expect_tx(&full[stage], stageBytes);
          armed |= 1u << stage;
          armed_par = (armed_par & ~(1u << stage)) | (phase << stage);
          // every term in one box per operand: term t lands t * kTcABytes (A) or t * bBytes
          // (B) after the operand's start
          const uint32_t sa = sbase + (uint32_t)stage * stageBytes;
          const uint32_t sb = sa + (uint32_t)a.nterms * kTcABytes;
          if constexpr (MODE == TC_SYNTH) {
            // A: Phi rows r0 + 64 sg .., column halves c0 / 64, c0 / 64 + 1
            tma_load_4d(sa, mA, 0, tl.r0 + kTcStageK * sg, tl.c0 >> 6, 0, &full[stage]);
            // B: slabs r0 / 32 + 2 sg, + 1, ring pairs n0 ..
            tma_load_4d(sb, mB, 0, tl.n0, tl.r0 / 32 + kTcSlabs * sg, 0, &full[stage]);
          } else {
            // A: G at problem mp, ring pairs 64 sg .., column halves c0 / 64, c0 / 64 + 1
            tma_load_5d(sa, mA, 0, tl.mp, kTcStageK * sg, tl.c0 >> 6, 0, &full[stage]);
            // B: Lambda_ana rows r0 + n0 .., ring-pair blocks 2 sg, 2 sg + 1
            tma_load_4d(sb, mB, 0, tl.r0 + tl.n0, kTcSlabs * sg, 0, &full[stage]);
          }
          if (++stage == S) {
            stage = 0;
            phase ^= 1;
          }
        }
      }
      if (!ok) {
        // let the copies already issued land before the CTA unwinds (bounded)
        for (int s = 0; s < S; ++s) {
          if (!(armed >> s & 1u)) continue;
          const uint32_t par = (armed_par >> s) & 1u;
          for (uint32_t i = 0; i < kTcWaitLimit && !mbar_try_wait(&full[s], par); ++i) {
          }
        }
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    // ------------------------------------------------------------------ MMA issuer
    // Lane 0 alone walks the loop, waits, issues and commits.
    if (lane == 0) {
      // A: MN-major, 128B swizzle, halves 64 k x 128 B apart; B: K-major, 64B swizzle
      const uint64_t da0 = sdesc(sbase, (uint32_t)kTcStageK * 128u, 1024, 2);
      const uint64_t db0 = sdesc(sbase + (uint32_t)a.nterms * kTcABytes, 16, 512, 4);
      const uint32_t bterm16 = bBytes >> 4, bslab16 = ((uint32_t)a.nmax * 64u) >> 4;
      int stage = 0;
      uint32_t phase = 0;
      int acc = 0;
      uint32_t aphase = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < a.ntiles && ok; t += gridDim.x) {
        const TcTile tl = a.tiles[t];
        if (!mbar_wait_fast(&tempty[acc], aphase ^ 1, a.err, 2)) break;
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)acc * (uint32_t)(a.split ? 2 * a.cols : a.cols);
        const uint32_t idesc = idesc_bf16(tl.nsize);
        const int nst = (tl.nkb + kTcSlabs - 1) / kTcSlabs, sg0 = tl.kb0 / kTcSlabs;
        for (int sg = sg0; sg < nst; ++sg) {
          if (!mbar_wait_fast(&full[stage], phase, a.err, 3)) {
            ok = false;
            break;
          }
          tc_fence_after();
          {
            const uint32_t so = (uint32_t)stage * (stageBytes >> 4);
            const uint64_t da = da0 + so, db = db0 + so;
            const bool first = sg == sg0;
            const int nh = min(kTcSlabs, tl.nkb - kTcSlabs * sg);
            const uint32_t dc = d + (uint32_t)a.cols;
            if (a.nterms == 2) {
              if (a.split) issue_stage<2, true>(da, db, bterm16, bslab16, nh, d, dc, idesc, first);
              else issue_stage<2, false>(da, db, bterm16, bslab16, nh, d, dc, idesc, first);
            } else {
              if (a.split) issue_stage<3, true>(da, db, bterm16, bslab16, nh, d, dc, idesc, first);
              else issue_stage<3, false>(da, db, bterm16, bslab16, nh, d, dc, idesc, first);
            }
            tc_commit(&empty[stage]);
          }
          if (++stage == S) {
            stage = 0;
            phase ^= 1;
          }
        }
        if (!ok) break;
        tc_commit(&tfull[acc]);
        if (++acc == a.nbuf) {
          acc = 0;
          aphase ^= 1;
        }
      }
      // every MMA this thread issued has completed before TMEM is released (bounded)
      tc_commit(drain);
      for (uint32_t i = 0; i < kTcWaitLimit && !mbar_try_wait(drain, 0); ++i) {
      }
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------------ epilogue
    const int q = warp & 3;         // TMEM lane quadrant this warp may access
    const int h = (warp - 2) >> 2;  // which of the quadrant's warps: chunks h, h + kEpiPerQuad, ..
    int acc = 0;
    uint32_t aphase = 0, ephase = 0;
    for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
      const TcTile tl = a.tiles[t];
      // this tile's instance, copied into registers (stores through F or part could alias it)
      if (!mbar_wait(&tfull[acc], aphase, a.err, 4)) break;
      tc_fence_after();
      // this tile's instance: with one instance its fields are read from the kernel
      // parameters where they are used (constant-bank operands: measurably faster in the
      // store loop than register copies); with several they are copied into registers
      // once per tile (stores through F or part could alias the array)
      TcInst mi;
      if constexpr (MULTI) {
        // only the fields this launch's mode reads (fewer live registers)
        const TcInst* Ip = a.insts + tl.inst;
        mi.L = Ip->L, mi.nr = Ip->nr;
        if constexpr (MODE == TC_SYNTH) {
          mi.npairs = Ip->npairs;
        } else {
          mi.part = Ip->part, mi.q2 = Ip->q2, mi.nalm = Ip->nalm;
        }
      }
      const TcInst& I = MULTI ? mi : a.one;
      const int L = I.L, nr = I.nr;
      const int m = tl.mp >> 1, p = tl.mp & 1;
      const int c = tl.c0 + 32 * q + lane;
      const bool cvalid = c < 2 * nr;
      const uint32_t tacc = tmem + (uint32_t)acc * (uint32_t)(a.split ? 2 * a.cols : a.cols) + ((uint32_t)(32 * q) << 16);
      if constexpr (MODE == TC_SYNTH) {
        // F (FP32, ring-pair-major F[jp][mp][Cpad]) in 16-column chunks, spread over the
        // quadrant's warps; TMEM is released after each warp's last load, before its stores
        const int nch = (tl.nsize + 15) / 16;
        const int last = nch - 1 < h ? -1 : h + (nch - 1 - h) / kEpiPerQuad * kEpiPerQuad;
        if (last < 0) {
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&tempty[acc]);
        }
        // the chunk (32 columns x 16 ring pairs) goes through the warp's 2 KB of shared memory
        // and out by one tensor store, which keeps the F writes off the load/store path
        float* fst = red + (size_t)(warp - 2) * 512;
        const CUtensorMap* mF = MULTI ? c_tc_maps + 3 * tl.inst + 2 : &a.one.tmF;
        for (int ch = h; ch < nch; ch += kEpiPerQuad) {
          float v[16];
          tmem_ld16(tacc + (uint32_t)(ch * 16), v);
          if (a.split) {
            float w[16];
            tmem_ld16(tacc + (uint32_t)(ch * 16) + (uint32_t)a.cols, w);
#pragma unroll
            for (int j = 0; j < 16; ++j) v[j] += w[j];
          }
          if (ch == last) {
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[acc]);
          }
          if (lane == 0) bulk_wait_read();  // the previous chunk's box has left the buffer
          __syncwarp();
          // ring pairs below the tile's jz are written as zeros (their lambda are negligible)
#pragma unroll
          for (int j = 0; j < 16; ++j) fst[j * 32 + lane] = tl.n0 + ch * 16 + j < tl.jz ? 0.f : v[j];  // box order: [16 ring pairs][32 c]
          fence_proxy_async();
          __syncwarp();
          // a box that starts past the last ring pair holds no row: not issued (a box that
          // runs past it is clipped by the copy engine)
          if (lane == 0 && tl.n0 + ch * 16 < I.npairs) {
            tma_store_3d(mF, tl.c0 + 32 * q, tl.mp, tl.n0 + ch * 16, smem_u32(fst));
            bulk_commit();
          }
        }
        if (++acc == a.nbuf) {
          acc = 0;
          aphase ^= 1;
        }
        continue;
      }
      // TC_ANA_STORE takes 32-column chunks; the quadrature takes 16-column half chunks, so that
      // a 128-degree tile's eight halves spread 3, 3, 2 over a quadrant's three warps (whole
      // chunks would spread 2, 1, 1)
      const int cw = MODE == TC_ANA_STORE ? 32 : 16;
      const int nch = (tl.nsize + cw - 1) / cw;
      const int last = nch - 1 < h ? -1 : h + (nch - 1 - h) / kEpiPerQuad * kEpiPerQuad;  // this warp's last chunk
      if (last < 0) {
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&tempty[acc]);
      }
      for (int ch = h; ch < nch; ch += kEpiPerQuad) {
        const uint32_t ta = tacc + (uint32_t)(ch * cw);
        if constexpr (MODE == TC_ANA_STORE) {
          float v[32];
          tmem_ld32(ta, v);
          if (a.split) {
            float w[32];
            tmem_ld32(ta + (uint32_t)a.cols, w);
#pragma unroll
            for (int j = 0; j < 32; ++j) v[j] += w[j];
          }
          if (ch == last) {
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[acc]);
          }
          if (cvalid) {
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              const int k = tl.n0 + ch * 32 + j;
              if (ch * 32 + j < tl.nsize && k < tl.kvalid) {
                const int l = m + p + 2 * k;
                const int64_t o = alm_idx(l, m, L) * (2 * nr) + c;
                if (a.store_f32) ((float*)a.alm_out)[o] = v[j];
                else a.alm_out[o] = (double)v[j];
              }
            }
          }
          continue;
        }
        // radial quadrature (Eq. 5): sum over the shells of this tile of q^X_l[i] Phi_NL,lm(r_i), in
        // double-float.  The half chunk (the warp's 32 columns = 16 shells x (re, im), by 16
        // degrees) is turned around through the warp's scratch 8 degrees at a time (element
        // (d, col) at d 32 + (col ^ 2 d): no bank conflicts either way).  Lane (d, f, b) then sums,
        // for degree d and field f (T, E), shells 8 b .. 8 b + 7 of the warp's 16, re and im, one
        // after another: each product exactly as p + e (q = qh + ql: p = v qh rounded, e = its
        // rounding error by fmaf plus v ql), the p's by error-free two-sums, the e's plainly; the
        // two shell halves are joined across the lane pair at the end.  The weights of the 16
        // degrees are requested together, right after the accumulator columns are read.
        const int s0 = (tl.c0 >> 1) + 16 * q;  // shell of the warp's first column
        const int d = lane >> 2, f = (lane >> 1) & 1, b = lane & 1;
        float* scr = red + (size_t)4 * a.nmax * 8 + (size_t)(warp - 2) * 256;
        {
          float v[16];
          tmem_ld16(ta, v);
          if (a.split) {
            float w[16];
            tmem_ld16(ta + (uint32_t)a.cols, w);
#pragma unroll
            for (int j = 0; j < 16; ++j) v[j] += w[j];
          }
          if (ch == last) {
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[acc]);
          }
          float4 qq[2][4];  // [sub-block][shell pair]: (qh, ql) of two shells
#pragma unroll
          for (int sb = 0; sb < 2; ++sb) {
            const int jj = ch * 16 + sb * 8 + d;
            const int k = tl.n0 + jj;
            const bool dvalid = jj < tl.nsize && k < tl.kvalid;
            const float4* qrow =
                (const float4*)(I.q2 + ((size_t)(m + p + 2 * (dvalid ? k : 0)) * 2 + f) * ((nr + 1) & ~1) + s0 + 8 * b);
#pragma unroll
            for (int e = 0; e < 4; ++e)
              qq[sb][e] = (dvalid && s0 + 8 * b + 2 * e < nr) ? qrow[e] : make_float4(0.f, 0.f, 0.f, 0.f);
          }
#pragma unroll
          for (int sb = 0; sb < 2; ++sb) {
            __syncwarp();
#pragma unroll
            for (int dd = 0; dd < 8; ++dd) scr[dd * 32 + (lane ^ (2 * dd))] = v[sb * 8 + dd];
            __syncwarp();
            float hr = 0.f, lr = 0.f, hi = 0.f, li = 0.f;  // re and im, double-float
#pragma unroll
            for (int e = 0; e < 8; ++e) {
              const int col = 2 * (8 * b + e);
              const float xr = scr[d * 32 + (col ^ (2 * d))];
              const float xi = scr[d * 32 + ((col + 1) ^ (2 * d))];
              const float qh = (e & 1) ? qq[sb][e >> 1].z : qq[sb][e >> 1].x;
              const float ql = (e & 1) ? qq[sb][e >> 1].w : qq[sb][e >> 1].y;
              const float pr = xr * qh, pi = xi * qh;
              const float er = fmaf(xr, ql, fmaf(xr, qh, -pr)), ei = fmaf(xi, ql, fmaf(xi, qh, -pi));
              float sum, err;
              two_sum(hr, pr, sum, err);
              hr = sum;
              lr += err + er;
              two_sum(hi, pi, sum, err);
              hi = sum;
              li += err + ei;
            }
            // join the two shell halves (lanes b = 0, 1)
            {
              const float ohr = __shfl_xor_sync(0xffffffffu, hr, 1), olr = __shfl_xor_sync(0xffffffffu, lr, 1);
              const float ohi = __shfl_xor_sync(0xffffffffu, hi, 1), oli = __shfl_xor_sync(0xffffffffu, li, 1);
              float sum, err;
              two_sum(hr, ohr, sum, err);
              hr = sum;
              lr += olr + err;
              two_sum(hi, ohi, sum, err);
              hi = sum;
              li += oli + err;
            }
            const int jj = ch * 16 + sb * 8 + d;  // degree column within the tile
            if (jj < tl.nsize) {
              // lane b = 0 writes re, lane b = 1 im: red[q][jj][f][part][hi, lo]
              float* o = red + (size_t)q * (a.nmax * 8) + (size_t)jj * 8 + f * 4 + b * 2;
              o[0] = b ? hi : hr;
              o[1] = b ? li : lr;
            }
          }
        }
      }
      if constexpr (MODE == TC_ANA_QUAD) {
        if (!epi_sync(&epib[0], ephase, lane, a.err)) break;
        const int tid = threadIdx.x - 64;
        for (int n = tid; n < tl.nsize; n += 32 * kEpiWarps) {
          const int k = tl.n0 + n;
          if (k >= tl.kvalid) continue;
          // the four quadrants' double-float partials, summed as double-float (high parts by
          // error-free two-sums, low parts and rounding errors plainly) and widened to FP64 once
          // per value: 3 operations of the FP64 pipe per value instead of 16
          float sh[4], sl[4];  // T re, T im, E re, E im
#pragma unroll
          for (int f = 0; f < 4; ++f) sh[f] = red[(size_t)n * 8 + 2 * f], sl[f] = red[(size_t)n * 8 + 2 * f + 1];
#pragma unroll
          for (int w = 1; w < 4; ++w) {
            const float* rw = red + (size_t)w * (a.nmax * 8) + (size_t)n * 8;
#pragma unroll
            for (int f = 0; f < 4; ++f) {
              float sum, err;
              two_sum(sh[f], rw[2 * f], sum, err);
              sh[f] = sum;
              sl[f] += err + rw[2 * f + 1];
            }
          }
          double s[4];
#pragma unroll
          for (int f = 0; f < 4; ++f) s[f] = (double)sh[f] + (double)sl[f];
          const int l = m + p + 2 * k;
          double2* dst = I.part + ((size_t)(tl.c0 >> 7) * I.nalm + alm_idx(l, m, L)) * 2;
          dst[0] = make_double2(s[0], s[1]);
          dst[1] = make_double2(s[2], s[3]);
        }
        if (!epi_sync(&epib[1], ephase, lane, a.err)) break;
        ephase ^= 1;
      }
      if (++acc == a.nbuf) {
        acc = 0;
        aphase ^= 1;
      }
    }
  }

  if constexpr (MODE == TC_SYNTH) {
    if (warp >= 2 && lane == 0) bulk_wait_all();  // this warp's tensor stores are complete
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
  }
}

// The expiry path of the bounded waits, on its own: one thread waits, with `limit` tries, on
// an mbarrier whose phase nothing completes (count 1, no arrival), so the wait runs out,
// records code 6 in the error word and returns.  Used by the test hook fnl_test_wait_expiry.
__global__ void k_wait_probe(int* err, uint32_t limit) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  mbar_wait_n(&bar, 0, err, 6, limit);
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    FNL_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q));
    if (q != cudaDriverEntryPointSuccess || !p) throw Error(FNL_EUNSUPPORTED, "cuTensorMapEncodeTiled unavailable");
    fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  return fn;
}

}  // namespace

CUtensorMap make_tensor_map_f32(const void* base, int rank, const uint64_t* dims, const uint64_t* strides,
                                const uint32_t* box) {
  CUtensorMap m;
  uint32_t estr[5] = {1, 1, 1, 1, 1};
  CUresult r = encode_fn()(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, (cuuint32_t)rank, const_cast<void*>(base),
                           (const cuuint64_t*)dims, (const cuuint64_t*)strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) throw Error(FNL_ECUDA, "cuTensorMapEncodeTiled (FP32) failed with code " + std::to_string((int)r));
  return m;
}

CUtensorMap make_tensor_map_bf16(const void* base, int rank, const uint64_t* dims, const uint64_t* strides,
                                 const uint32_t* box, int swizzle_bytes) {
  CUtensorMap m;
  uint32_t estr[5] = {1, 1, 1, 1, 1};
  const CUtensorMapSwizzle sw = swizzle_bytes == 128  ? CU_TENSOR_MAP_SWIZZLE_128B
                                : swizzle_bytes == 64 ? CU_TENSOR_MAP_SWIZZLE_64B
                                                      : CU_TENSOR_MAP_SWIZZLE_NONE;
  CUresult r = encode_fn()(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, (cuuint32_t)rank, const_cast<void*>(base),
                           (const cuuint64_t*)dims, (const cuuint64_t*)strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) throw Error(FNL_ECUDA, "cuTensorMapEncodeTiled failed with code " + std::to_string((int)r));
  return m;
}

size_t tc_smem_bytes(int nterms, int nmax, int stages, int mode) {
  const size_t stage = (size_t)nterms * (kTcABytes + (size_t)nmax * 64 * kTcSlabs);
  // epilogue: per-warp 2 KB staging of F boxes (synthesis), or the quadrature's reduction and
  // per-warp scratch (analysis)
  const size_t red = mode == TC_SYNTH ? (size_t)kEpiWarps * 512 * sizeof(float)
                                      : ((size_t)4 * nmax * 8 + (size_t)kEpiWarps * 256) * sizeof(float);
  return 1024 /*alignment*/ + (size_t)stages * stage + 1024 /*barriers*/ + red;
}

int tc_stages(int nterms, int nmax, int mode) {
  int s = 6;
  while (s > 1 && tc_smem_bytes(nterms, nmax, s, mode) > 227 * 1024) --s;
  return s;
}

void upload_tc_maps(const CUtensorMap* host, int n, cudaStream_t st) {
  if (n < 1 || n > kTcMaxInst) throw Error(FNL_EINVAL, "too many instances for one tensor-core launch");
  FNL_CUDA(cudaMemcpyToSymbolAsync(c_tc_maps, host, sizeof(CUtensorMap) * 3 * (size_t)n, 0,
                                   cudaMemcpyHostToDevice, st));
}

void launch_wait_probe(int* err, uint32_t limit, cudaStream_t st) {
  k_wait_probe<<<1, 32, 0, st>>>(err, limit);
  FNL_CUDA(cudaGetLastError());
}

void launch_tc_gemm(const TcArgs& args, int sms, cudaStream_t st) {
  const size_t smem = tc_smem_bytes(args.nterms, args.nmax, args.stages, args.mode);
  if (smem > 227 * 1024 || args.stages < 1) throw Error(FNL_EUNSUPPORTED, "tensor-core tile does not fit shared memory");
  const int grid = std::max(1, std::min(args.ntiles, sms));
  auto run = [&](auto kern) {
    FNL_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<grid, kThreadsTc, smem, st>>>(args);
  };
  if (args.multi) {
    if (args.mode == TC_SYNTH) run(k_tc_gemm<true, TC_SYNTH>);
    else if (args.mode == TC_ANA_QUAD) run(k_tc_gemm<true, TC_ANA_QUAD>);
    else throw Error(FNL_EUNSUPPORTED, "per-shell analysis output runs for one configuration per launch");
  } else {
    if (args.mode == TC_SYNTH) run(k_tc_gemm<false, TC_SYNTH>);
    else if (args.mode == TC_ANA_QUAD) run(k_tc_gemm<false, TC_ANA_QUAD>);
    else run(k_tc_gemm<false, TC_ANA_STORE>);
  }
  FNL_CUDA(cudaGetLastError());
}

}  // namespace fnl
