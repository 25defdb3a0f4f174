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

struct TcArgs {
  CUtensorMap tmA[3];   // per BF16 term: Phi (synthesis) or G (analysis)
  CUtensorMap tmB[3];   // per BF16 term: Lambda_syn or Lambda_ana, boxes of bbox rows
  CUtensorMap tmB16[3]; // the same operands in 16-row boxes (tile remainders)
  const TcTile* tiles;
  int ntiles;
  int mode;
  int nterms;           // 2 or 3
  int split;            // 1: products of the leading terms and the correction products go to two
                        //    separate accumulators (tile width <= 128), summed in the epilogue
  int nmax;             // largest tile width in this launch (B stage size)
  int bbox;             // rows of one B box (multiple of 16)
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
size_t tc_smem_bytes(int nterms, int nmax, int stages);
int tc_stages(int nterms, int nmax);
void launch_tc_gemm(const TcArgs& args, int sms, cudaStream_t st);

}  // namespace fnl
