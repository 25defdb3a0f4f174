// Tensor-core Legendre GEMM of the mixed-precision forms (see tc_gemm.cu).
#pragma once

#include <cuda.h>

#include <cstdint>

namespace fnl {

enum TcMode { TC_SYNTH = 0, TC_ANA_QUAD = 1, TC_ANA_STORE = 2 };

// One output tile: problem mp = 2 m + p, column tile c0 (multiple of 128), N range
// [n0, n0 + nsize) (ring pairs for the synthesis, degrees k for the analysis), nkb
// 32-deep k blocks, r0 = first row of the problem in the packed operand, kvalid = K_mp,
// inst = the configuration (TcInst) the tile belongs to.  Ring pairs below the order's jmin
// (where every |lambda_lm| < 2^-30) are left out: the synthesis writes their rows of F as
// zeros (jz = jmin), and the analysis starts its k loop at the 32-deep block kb0 (the
// 64-ring-pair stage holding jmin).
struct TcTile {
  int mp, c0, n0, nsize, nkb, r0, kvalid, inst;
  int jz, kb0;
};

// Operands arrive in stages 64 deep in k: one TMA box of A holding every BF16 term (per term
// 128 columns x 64 k, both 64-column halves, MN-major, 128B swizzle) and one of B (per term
// nmax rows x 64 k as two 32-deep slabs, K-major, 64B swizzle), and one commit releases the
// stage.
constexpr int kTcStageK = 64;
constexpr int kTcSlabs = kTcStageK / 32;               // 32-deep B slabs per stage
constexpr uint32_t kTcABytes = 128u * kTcStageK * 2u;  // A bytes per term and stage

// Instances (configurations or realisations) in one multi-instance launch, at most.
constexpr int kTcMaxInst = 64;

// What differs between the instances that share one launch; an array of these lives in
// device memory and every tile names its entry.  The tensor maps are kept apart (kernel
// parameters for one instance, a constant-memory table for several): the copy engine reads
// a map from global memory far more slowly than from those two spaces.
struct alignas(128) TcInst {  // CUtensorMap is 128-byte aligned
  CUtensorMap tmA;      // Phi (synthesis) or G (analysis), box {64 c, 64 k, 2 halves, terms}
  CUtensorMap tmB;      // Lambda_syn or Lambda_ana, box {32 k, nmax rows, 2 slabs, terms}
  CUtensorMap tmF;      // TC_SYNTH: F as FP32 [npairs][nmp][Cpad], box {32 c, 1 problem, 16 ring
                        // pairs} for the epilogue's tensor stores
  float* F;             // TC_SYNTH: [npairs][nmp][Cpad] (ring-pair-major)
  double2* part;        // TC_ANA_QUAD: [Cpad / 128][nalm][2] ((T re, T im), (E re, E im))
  const float2* q2;     // [L+1][2][nre] q^T, q^E as FP32 pairs (hi, lo), nre = nr rounded up to even
  int L, nr, npairs, Cpad;
  int64_t nalm;
};

struct TcArgs {
  TcInst one;           // the single instance (multi == 0), maps and fields in parameter space
  int multi;            // 1: maps of instance i at c_tc_maps[3 i] (A), c_tc_maps[3 i + 1] (B) and
                        //    c_tc_maps[3 i + 2] (F), its other fields at insts[i]
  const TcInst* insts;  // device array indexed by TcTile::inst (multi == 1)
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
  double* alm_out;      // TC_ANA_STORE (one configuration per launch): [nalm][nr][2]
  int store_f32;        // TC_ANA_STORE: 1 writes those values as FP32 (the accumulators' own type)
  int* err;             // device error word (0 = ok)
};

CUtensorMap make_tensor_map_bf16(const void* base, int rank, const uint64_t* dims, const uint64_t* strides,
                                 const uint32_t* box, int swizzle_bytes);
// The same for an FP32 tensor, without swizzle.
CUtensorMap make_tensor_map_f32(const void* base, int rank, const uint64_t* dims, const uint64_t* strides,
                                const uint32_t* box);
size_t tc_smem_bytes(int nterms, int nmax, int stages, int mode);
int tc_stages(int nterms, int nmax, int mode);
void launch_tc_gemm(const TcArgs& args, int sms, cudaStream_t st);
// One bounded mbarrier wait that nothing completes, with `limit` tries (the expiry path).
void launch_wait_probe(int* err, uint32_t limit, cudaStream_t st);
// Copy n instances' maps (A, B and F each) into the constant table, on `st` from pinned
// host memory that stays unchanged until the copy has run.
void upload_tc_maps(const CUtensorMap* host, int n, cudaStream_t st);

}  // namespace fnl
