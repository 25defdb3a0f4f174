// Tensor-core Legendre GEMM of the mixed-precision forms (see tc_gemm.cu).
#pragma once

#include <cuda.h>

#include <cstdint>

namespace fnl {

enum TcMode { TC_SYNTH = 0, TC_ANA_QUAD = 1, TC_ANA_STORE = 2 };

// One output tile: problem mp = 2 m + p, column tile c0 (multiple of 128), N range
// [n0, n0 + nsize) (ring pairs for the synthesis, degrees k for the analysis), nkb
// 32-deep k blocks, r0 = first row of the problem in the packed operand, kvalid = K_mp.
struct TcTile {
  int mp, c0, n0, nsize, nkb, r0, kvalid, pad;
};

// Operands arrive in stages 64 deep in k: per BF16 term one TMA box of A (128 columns x 64 k,
// both 64-column halves, MN-major, 128B swizzle) and one of B (nmax rows x 64 k as two
// 32-deep slabs, K-major, 64B swizzle), and one commit releases the stage.
constexpr int kTcStageK = 64;
constexpr uint32_t kTcABytes = 128u * kTcStageK * 2u;  // A bytes per term and stage

struct TcArgs {
  CUtensorMap tmA[3];   // per BF16 term: Phi (synthesis) or G (analysis), box {64 c, 64 k, 2 halves}
  CUtensorMap tmB[3];   // per BF16 term: Lambda_syn or Lambda_ana, box {32 k, nmax rows, 2 slabs}
  const TcTile* tiles;
  int ntiles;
  int mode;
  int nterms;           // 2 or 3
  int split;            // 1: products of the leading terms and the correction products go to two
                        //    separate accumulators (tile width <= 128), summed in the epilogue
  int nmax;             // largest tile width in this launch (rows of every B box)
  int cols;             // TMEM columns between the leading and the correction accumulator
  int nbuf;             // accumulator sets in TMEM (double buffering when 2)
  int stages;
  int L, nr, npairs, Cpad;
  int64_t nalm;
  float* F;             // TC_SYNTH: [npairs][nmp][Cpad] (ring-pair-major)
  float4* part;         // TC_ANA_QUAD: [Cpad / 128][nalm] (T re, T im, E re, E im)
  double* alm_out;      // TC_ANA_STORE: [nalm][nr][2]
  const float* qT;      // [L+1][nr]
  const float* qE;
  int* err;             // device error word (0 = ok)
};

CUtensorMap make_tensor_map_bf16(const void* base, int rank, const uint64_t* dims, const uint64_t* strides,
                                 const uint32_t* box, int swizzle_bytes);
size_t tc_smem_bytes(int nterms, int nmax, int stages, int mode);
int tc_stages(int nterms, int nmax, int mode);
void launch_tc_gemm(const TcArgs& args, int sms, cudaStream_t st);

}  // namespace fnl
