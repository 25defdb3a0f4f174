// C ABI of libfnl: argument validation, set-up of the shells object and the entry points
// that chain the kernels of the path (Sect. 2, recipe steps (i)-(v)).
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <atomic>
#include <functional>
#include <string>
#include <vector>

#include "fnl_internal.cuh"

namespace fnl {

static thread_local std::string g_last_error;

void set_last_error(const std::string& msg) { g_last_error = msg; }

fnl_status guard(const std::function<void()>& body) {
  g_last_error.clear();
  try {
    body();
    return FNL_OK;
  } catch (const Error& e) {
    g_last_error = e.what();
    return e.code;
  } catch (const std::bad_alloc&) {
    g_last_error = "host allocation failed";
    return FNL_ENOMEM;
  } catch (const std::exception& e) {
    g_last_error = e.what();
    return FNL_EINVAL;
  } catch (...) {
    g_last_error = "unknown error";
    return FNL_EINVAL;
  }
}

DeviceScope::DeviceScope(int dev) {
  FNL_CUDA(cudaGetDevice(&prev));
  if (prev != dev) FNL_CUDA(cudaSetDevice(dev));
}
DeviceScope::~DeviceScope() {
  if (prev >= 0) cudaSetDevice(prev);
}

namespace {

bool smooth235(int n) {
  if (n < 1) return false;
  for (int p : {2, 3, 5})
    while (n % p == 0) n /= p;
  return n == 1;
}

}  // namespace

// Allocation-failure test hook: -1 = off; n >= 0 = the allocation after the next n ones fails
// (once; the hook then turns itself off).
static std::atomic<long> g_fail_alloc{-1};

void* device_malloc(size_t bytes) {
  long n = g_fail_alloc.load();
  while (n >= 0) {
    if (g_fail_alloc.compare_exchange_weak(n, n == 0 ? -1 : n - 1)) {
      if (n == 0) throw Error(FNL_ENOMEM, "device allocation failed (simulated by fnl_test_fail_alloc)");
      break;
    }
  }
  void* p = nullptr;
  FNL_CUDA(cudaMalloc(&p, bytes ? bytes : 1));
  return p;
}

void check_dev_ptr(const void* p, const char* name, bool nullable) {
  if (!p) {
    if (!nullable) throw Error(FNL_EINVAL, std::string(name) + " must not be NULL");
    return;
  }
  if (((uintptr_t)p) % 16 != 0) throw Error(FNL_EINVAL, std::string(name) + " must be 16-byte aligned");
  cudaPointerAttributes attr;
  cudaError_t e = cudaPointerGetAttributes(&attr, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    throw Error(FNL_EINVAL, std::string(name) + " is not a pointer CUDA knows");
  }
  if (attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged)
    throw Error(FNL_EINVAL, std::string(name) + " must be device memory");
}

void check_shells(const fnl_shells* sh) {
  if (!sh) throw Error(FNL_EINVAL, "shells object is NULL");
}

namespace {

template <typename T>
T* dalloc(fnl_shells* sh, size_t count) {
  const size_t bytes = sizeof(T) * (count ? count : 1);
  void* p = device_malloc(bytes);
  sh->allocations.push_back(p);
  sh->device_bytes += bytes;
  return (T*)p;
}

template <typename T>
T* upload(fnl_shells* sh, const std::vector<T>& v) {
  T* p = dalloc<T>(sh, v.size());
  FNL_CUDA(cudaMemcpy(p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice));
  return p;
}

void free_shells(fnl_shells* sh) {
  if (!sh) return;
  for (auto& e : sh->ring)
    if (e) cudaEventDestroy(e);
  for (void* p : sh->allocations) cudaFree(p);
  sh->allocations.clear();
  delete sh;
}

void validate_desc(const fnl_shell_desc* d, bool synth_only = false, bool healpix = false) {
  FNL_REQUIRE(d, "desc is NULL");
  FNL_REQUIRE(d->lmax >= 1 && d->lmax <= 4096, "lmax must be in [1, 4096]");
  FNL_REQUIRE(d->nr >= 1 && d->nr <= (synth_only ? 256 : 128), "nr must be in [1, 128]");
  FNL_REQUIRE(healpix || d->ntheta >= d->lmax + 1, "ntheta must be >= lmax + 1");
  FNL_REQUIRE(healpix || d->nphi >= 2 * d->lmax + 2, "nphi must be >= 2 lmax + 2");
  FNL_REQUIRE(smooth235(d->nphi), "nphi must be 2/3/5-smooth");
  FNL_REQUIRE(d->r && d->w, "r and w must not be NULL");
  FNL_REQUIRE(d->alphaT && d->alphaE, "alphaT and alphaE must not be NULL");
  FNL_REQUIRE(d->prec >= FNL_FP64 && d->prec <= FNL_BF16X3, "unknown precision");
  if (!d->K && !synth_only) {
    FNL_REQUIRE(d->nk >= 2, "nk must be >= 2");
    FNL_REQUIRE(d->kmin > 0 && d->kmax > d->kmin, "need 0 < kmin < kmax");
    FNL_REQUIRE(d->A > 0 && std::isfinite(d->ns), "need A > 0 and finite ns");
    FNL_REQUIRE(d->jitter_rel >= 0, "jitter_rel must be >= 0");
    for (int i = 0; i < d->nr; ++i) FNL_REQUIRE(d->r[i] > 0, "r_i must be > 0");
  }
  const size_t tsize = d->prec == FNL_FP64 ? sizeof(double) : sizeof(float);
  FNL_REQUIRE(2 * 2 * tsize * (size_t)d->nphi <= 200 * 1024, "nphi too large for the shared-memory ring FFT");
}

// Tables, scratch, tile lists and tensor maps of the tensor-core forms.
void setup_mixed(fnl_shells* sh, const std::vector<double>& qT, const std::vector<double>& qE) {
  const int L = sh->lmax, nr = sh->nr, np = sh->npairs, nmp = 2 * (L + 1), T = sh->nterms;
  const int Cpad = sh->Cpad;
  const int64_t rows32 = sh->row32[nmp], rows16 = sh->rows_total, nslab = rows32 / 32;
  typedef unsigned short bf16_t;
  sh->phiT_stride = rows32 * Cpad;
  sh->d_phiT = dalloc<bf16_t>(sh, (size_t)T * sh->phiT_stride);
  sh->lsyn_stride = nslab * np * 32;
  sh->d_lsyn = dalloc<bf16_t>(sh, (size_t)T * sh->lsyn_stride);
  sh->lana_stride = rows16 * sh->npj;
  sh->d_lana = dalloc<bf16_t>(sh, (size_t)T * sh->lana_stride);
  sh->gt_stride = (int64_t)nmp * np * Cpad;
  sh->d_GT = dalloc<bf16_t>(sh, (size_t)T * sh->gt_stride);
  sh->d_F = dalloc<float>(sh, (size_t)nmp * np * Cpad);
  sh->d_part = dalloc<double>(sh, 4 * (size_t)(Cpad / 128) * sh->nalm);
  sh->d_err = dalloc<int>(sh, 1);
  sh->d_psum = dalloc<double>(sh, nr);
  sh->d_psum_part = dalloc<double>(sh, (size_t)(L + 1) * 2 * nr);
  FNL_CUDA(cudaMemset(sh->d_phiT, 0, sizeof(bf16_t) * (size_t)T * sh->phiT_stride));
  FNL_CUDA(cudaMemset(sh->d_lsyn, 0, sizeof(bf16_t) * (size_t)T * sh->lsyn_stride));
  FNL_CUDA(cudaMemset(sh->d_lana, 0, sizeof(bf16_t) * (size_t)T * sh->lana_stride));
  FNL_CUDA(cudaMemset(sh->d_GT, 0, sizeof(bf16_t) * (size_t)T * sh->gt_stride));
  FNL_CUDA(cudaMemset(sh->d_F, 0, sizeof(float) * (size_t)nmp * np * Cpad));
  FNL_CUDA(cudaMemset(sh->d_err, 0, sizeof(int)));
  // q^T, q^E of the quadrature epilogue as FP32 pairs hi + lo (48 significant bits), [l][X][i],
  // rows of an even number of shells (zero-padded) so that the epilogue's 16-byte loads of two
  // shells stay aligned
  const int nre = (nr + 1) & ~1;
  std::vector<float> q2((size_t)(L + 1) * 2 * nre * 2, 0.f);
  for (int l = 0; l <= L; ++l)
    for (int X = 0; X < 2; ++X)
      for (int i = 0; i < nr; ++i) {
        const double v = (X ? qE : qT)[(size_t)l * nr + i];
        const float hi = (float)v;
        const size_t o = (((size_t)l * 2 + X) * nre + i) * 2;
        q2[o] = hi;
        q2[o + 1] = (float)(v - (double)hi);
      }
  sh->d_q2 = (float2*)upload(sh, q2);
  sh->d_row32 = upload(sh, sh->row32);
  {
    std::vector<float> tw2, tw1;
    ring_square_tables(sh->nphi, tw2, tw1);
    if (!tw2.empty()) {
      sh->d_sqtw2 = upload(sh, tw2);
      sh->d_sqtw1 = upload(sh, tw1);
    }
  }
  build_lambda_tables_mixed(sh, 0);

  // tile lists: capacity for the narrowest tiles configure_tc accepts, then the default shapes
  {
    int64_t cap_syn = 0, cap_ana = 0;
    for (int mp = 0; mp < nmp; ++mp) {
      const int K = sh->K[mp];
      if (!K) continue;
      cap_syn += (int64_t)((np + kTcMinWidth - 1) / kTcMinWidth) * (Cpad / 128);
      cap_ana += (int64_t)((K + kTcMinWidth - 1) / kTcMinWidth) * (Cpad / 128);
    }
    sh->d_tc_syn = dalloc<TcTile>(sh, (size_t)cap_syn);
    sh->d_tc_ana = dalloc<TcTile>(sh, (size_t)cap_ana);
  }
  sh->d_tci = dalloc<TcInst>(sh, 2);
  build_tc_inst_a(sh);
  for (TcArgs* a : {&sh->tc_syn, &sh->tc_ana}) {
    a->nterms = T;
    a->split = sh->tc_split;
    a->alm_out = nullptr;
    a->store_f32 = 0;
    a->err = sh->d_err;
  }
  sh->tc_syn.insts = sh->d_tci;
  sh->tc_ana.insts = sh->d_tci + 1;
  sh->tc_syn.mode = TC_SYNTH;
  sh->tc_ana.mode = TC_ANA_QUAD;
  configure_tc(sh, 256, 256);
}

}  // namespace

// Tensor map of an F buffer (FP32 [npairs][nmp][Cpad]) for the synthesis epilogue's tensor
// stores: boxes of 32 columns x 1 problem x 16 ring pairs.
CUtensorMap f_tensor_map(const fnl_shells* sh, const void* F) {
  const int nmp = 2 * (sh->lmax + 1);
  const uint64_t dims[3] = {(uint64_t)sh->Cpad, (uint64_t)nmp, (uint64_t)sh->npairs};
  const uint64_t str[2] = {(uint64_t)sh->Cpad * 4, (uint64_t)nmp * sh->Cpad * 4};
  const uint32_t box[3] = {32, 1, 16};
  return make_tensor_map_f32(F, 3, dims, str, box);
}

// The per-configuration part of the tensor-core GEMMs' arguments that does not depend on
// the tile shape: the A tensor maps (BF16, MN-major, 128B swizzle; boxes of 64 columns x 64 k
// x both 64-column halves of a 128-column tile, through a view whose next dimension steps over
// the halves, 128 B apart, and whose last dimension steps over the BF16 terms) and the scratch
// and table pointers.  Entry 0 is the synthesis, entry 1 the analysis.
void build_tc_inst_a(fnl_shells* sh) {
  const int L = sh->lmax, nr = sh->nr, np = sh->npairs, nmp = 2 * (L + 1), T = sh->nterms, Cpad = sh->Cpad;
  const int64_t rows32 = sh->row32[nmp];
  {
    const uint64_t dims[4] = {64, (uint64_t)rows32, (uint64_t)Cpad / 64, (uint64_t)T};
    const uint64_t str[3] = {(uint64_t)Cpad * 2, 128, (uint64_t)sh->phiT_stride * 2};
    const uint32_t box[4] = {64, (uint32_t)kTcStageK, 2, (uint32_t)T};
    sh->tci[0].tmA = make_tensor_map_bf16(sh->d_phiT, 4, dims, str, box, 128);
  }
  {
    // G is ring-pair-major, [term][jp][mp][Cpad]: box of 64 columns x 1 problem x 64 ring pairs
    // x 2 halves x every term
    const uint64_t dims[5] = {64, (uint64_t)nmp, (uint64_t)np, (uint64_t)Cpad / 64, (uint64_t)T};
    const uint64_t str[4] = {(uint64_t)Cpad * 2, (uint64_t)nmp * Cpad * 2, 128, (uint64_t)sh->gt_stride * 2};
    const uint32_t box[5] = {64, 1, (uint32_t)kTcStageK, 2, (uint32_t)T};
    sh->tci[1].tmA = make_tensor_map_bf16(sh->d_GT, 5, dims, str, box, 128);
  }
  sh->tci[0].tmF = f_tensor_map(sh, sh->d_F);
  for (TcInst& I : sh->tci) {
    I.F = (float*)sh->d_F;
    I.part = (double2*)sh->d_part;
    I.q2 = sh->d_q2;
    I.L = L;
    I.nr = nr;
    I.npairs = np;
    I.Cpad = Cpad;
    I.nalm = sh->nalm;
  }
}

// Tensor maps of the B operands (BF16, K-major, 64B swizzle): boxes of nmax rows x two 32-deep
// slabs (64 k per stage) x every BF16 term; rows past the table are zero-filled.  Then the
// two entries go to the device.
void build_tc_inst_b(fnl_shells* sh) {
  const int L = sh->lmax, np = sh->npairs, nmp = 2 * (L + 1), T = sh->nterms;
  const int64_t nslab = sh->row32[nmp] / 32, rows16 = sh->rows_total;
  {
    // Lambda_syn [term][slab][jp][32 k]
    const uint64_t dims[4] = {32, (uint64_t)np, (uint64_t)nslab, (uint64_t)T};
    const uint64_t str[3] = {64, (uint64_t)np * 64, (uint64_t)sh->lsyn_stride * 2};
    const uint32_t box[4] = {32, (uint32_t)sh->tc_syn.nmax, (uint32_t)kTcSlabs, (uint32_t)T};
    sh->tci[0].tmB = make_tensor_map_bf16(sh->d_lsyn, 4, dims, str, box, 64);
  }
  {
    // Lambda_ana [term][row16][npj]: 32 ring pairs x rows x blocks of 32 ring pairs (64 B
    // apart; npj is a multiple of 32, so every block stays inside its row)
    const uint64_t dims[4] = {32, (uint64_t)rows16, (uint64_t)sh->npj / 32, (uint64_t)T};
    const uint64_t str[3] = {(uint64_t)sh->npj * 2, 64, (uint64_t)sh->lana_stride * 2};
    const uint32_t box[4] = {32, (uint32_t)sh->tc_ana.nmax, (uint32_t)kTcSlabs, (uint32_t)T};
    sh->tci[1].tmB = make_tensor_map_bf16(sh->d_lana, 4, dims, str, box, 64);
  }
  FNL_CUDA(cudaMemcpy(sh->d_tci, sh->tci, sizeof(sh->tci), cudaMemcpyHostToDevice));
  sh->tc_syn.one = sh->tci[0];
  sh->tc_ana.one = sh->tci[1];
  sh->tc_syn.multi = sh->tc_ana.multi = 0;
}

// Tile shapes of the two tensor-core GEMMs.  Synthesis tiles are `nsyn` ring pairs wide, the
// width <= syn_cap that wastes the fewest ring pairs (each tile charged 16 columns of
// overhead); analysis tiles cover up to `ana_cap` degrees.  Both caps are multiples of 16 in
// [kTcMinWidth, 256].  Products of the leading terms and the correction products accumulate
// in two separate accumulators `cols` apart; as many accumulator sets as fit in the 512 TMEM
// columns (at most 2) rotate over tiles, so 128-wide tiles double-buffer the epilogue and
// 256-wide tiles issue half as many, wider MMAs.  The shape changes no result: every output
// element sums its k blocks in the same order whatever the tiling.
void configure_tc(fnl_shells* sh, int syn_cap, int ana_cap, bool exact) {
  FNL_REQUIRE(syn_cap >= kTcMinWidth && syn_cap <= 256 && syn_cap % 16 == 0 && ana_cap >= kTcMinWidth &&
                  ana_cap <= 256 && ana_cap % 16 == 0,
              "tile widths must be multiples of 16 in [64, 256]");
  const int L = sh->lmax, np = sh->npairs, nmp = 2 * (L + 1), T = sh->nterms;
  int best = syn_cap, bestc = 1 << 30;
  for (int n = syn_cap; n >= kTcMinWidth && !exact; n -= 16) {
    const int tiles = (np + n - 1) / n, cost = tiles * (n + 16);
    if (cost < bestc) {
      bestc = cost;
      best = n;
    }
  }
  sh->nsyn = best;
  sh->nana = ana_cap;
  const int ctiles = sh->Cpad / 128;
  std::vector<TcTile> ts, ta;
  for (int mp = 0; mp < nmp; ++mp) {
    const int K = sh->K[mp];
    if (!K) continue;
    // ring pairs below jmin carry only |lambda| < kLambdaSkip for this order: synthesis tiles
    // wholly below it are left out (F keeps its zeros there) and the others write zeros there;
    // the analysis k loop starts at the 64-ring-pair stage holding jmin
    const int jz = sh->jmin.empty() ? 0 : sh->jmin[mp / 2];
    const int kb0 = std::min(jz / kTcStageK, ((np + 31) / 32 - 1) / kTcSlabs) * kTcSlabs;  // >= 1 stage left
    for (int n0 = 0; n0 < np; n0 += sh->nsyn) {
      if (n0 + sh->nsyn <= jz) continue;
      for (int ct = 0; ct < ctiles; ++ct)
        ts.push_back({mp, 128 * ct, n0, sh->nsyn, (K + 31) / 32, (int)sh->row32[mp], K, 0, jz, 0});
    }
    for (int n0 = 0; n0 < K;) {
      const int n = std::min(ana_cap, round_up(K - n0, 16));
      for (int ct = 0; ct < ctiles; ++ct)
        ta.push_back({mp, 128 * ct, n0, n, (np + 31) / 32, (int)sh->row0[mp], K, 0, 0, kb0});
      n0 += n;
    }
  }
  // largest problems first (the CTAs take tiles round robin), but the tiles of one problem
  // stay adjacent: they share its operand slab (Phi or G rows, Lambda rows across column
  // tiles), which then comes from L2 instead of DRAM for all but the first of them
  auto group_sort = [](std::vector<TcTile>& v) {
    std::vector<std::pair<int64_t, int>> groups;  // (cost, first index) per problem
    for (size_t i = 0; i < v.size(); ++i) {
      if (i == 0 || v[i].mp != v[i - 1].mp) groups.push_back({0, (int)i});
      groups.back().first += (int64_t)(v[i].nkb - v[i].kb0) * v[i].nsize;
    }
    std::stable_sort(groups.begin(), groups.end(), [](const auto& a, const auto& b) { return a.first > b.first; });
    std::vector<TcTile> out;
    out.reserve(v.size());
    for (const auto& g : groups)
      for (size_t i = g.second; i < v.size() && v[i].mp == v[g.second].mp; ++i) out.push_back(v[i]);
    v.swap(out);
  };
  group_sort(ts);
  group_sort(ta);
  FNL_CUDA(cudaMemcpy(sh->d_tc_syn, ts.data(), sizeof(TcTile) * ts.size(), cudaMemcpyHostToDevice));
  FNL_CUDA(cudaMemcpy(sh->d_tc_ana, ta.data(), sizeof(TcTile) * ta.size(), cudaMemcpyHostToDevice));
  int widest_ana = 16;
  for (const TcTile& t : ta) widest_ana = std::max(widest_ana, t.nsize);
  if (exact) widest_ana = ana_cap;  // every configuration of a multi-instance launch: the same box
  sh->tiles_syn_h = ts;
  sh->tiles_ana_h = ta;
  ++sh->tiles_version;
  for (TcArgs* a : {&sh->tc_syn, &sh->tc_ana}) {
    const bool syn = a == &sh->tc_syn;
    const int nm = syn ? sh->nsyn : widest_ana;
    a->cols = nm <= 128 ? 128 : 256;
    a->nbuf = std::min(2, 512 / (a->split ? 2 * a->cols : a->cols));
    a->nmax = nm;
    a->stages = tc_stages(T, nm, a->mode);
    a->tiles = syn ? sh->d_tc_syn : sh->d_tc_ana;
    a->ntiles = (int)(syn ? ts.size() : ta.size());
  }
  build_tc_inst_b(sh);
}

fnl_shells* clone_scratch(const fnl_shells* src) {
  FNL_REQUIRE(src->nterms, "scratch clones are made for the tensor-core forms");
  DeviceScope scope(src->device);
  fnl_shells* c = new fnl_shells(*src);
  c->allocations.clear();
  c->device_bytes = 0;
  c->ring.clear();
  c->ring_slots = c->ring_head = c->ring_count = 0;
  c->owner = src->owner ? src->owner : src;
  c->maps_ready = false;
  c->d_mapL = c->d_mapW = c->d_mapX = c->d_Fiqu = nullptr;
  c->d_maps_jmin = nullptr;
  try {
    typedef unsigned short bf16_t;
    const int L = c->lmax, nr = c->nr, np = c->npairs, nmp = 2 * (L + 1), T = c->nterms, Cpad = c->Cpad;
    c->d_phiT = dalloc<bf16_t>(c, (size_t)T * c->phiT_stride);
    c->d_GT = dalloc<bf16_t>(c, (size_t)T * c->gt_stride);
    c->d_F = dalloc<float>(c, (size_t)nmp * np * Cpad);
    c->d_part = dalloc<double>(c, 4 * (size_t)(Cpad / 128) * c->nalm);
    c->d_err = dalloc<int>(c, 1);
    c->d_psum = dalloc<double>(c, nr);
    c->d_psum_part = dalloc<double>(c, (size_t)(L + 1) * 2 * nr);
    c->d_aL = dalloc<double>(c, 4 * (size_t)c->nalm);
    c->d_aNL = dalloc<double>(c, 4 * (size_t)c->nalm);
    c->d_aOut = dalloc<double>(c, 4 * (size_t)c->nalm);
    c->d_tci = dalloc<TcInst>(c, 2);
    FNL_CUDA(cudaMemset(c->d_phiT, 0, sizeof(bf16_t) * (size_t)T * c->phiT_stride));
    FNL_CUDA(cudaMemset(c->d_GT, 0, sizeof(bf16_t) * (size_t)T * c->gt_stride));
    FNL_CUDA(cudaMemset(c->d_F, 0, sizeof(float) * (size_t)nmp * np * Cpad));
    FNL_CUDA(cudaMemset(c->d_err, 0, sizeof(int)));
    build_tc_inst_a(c);
    refresh_clone(c, src);
  } catch (...) {
    free_shells(c);
    throw;
  }
  return c;
}

void refresh_clone(fnl_shells* c, const fnl_shells* src) {
  for (int k = 0; k < 2; ++k) c->tci[k].tmB = src->tci[k].tmB;
  FNL_CUDA(cudaMemcpy(c->d_tci, c->tci, sizeof(c->tci), cudaMemcpyHostToDevice));
  c->tc_syn = src->tc_syn;
  c->tc_ana = src->tc_ana;
  c->tc_syn.one = c->tci[0];
  c->tc_ana.one = c->tci[1];
  c->tc_syn.insts = c->d_tci;
  c->tc_ana.insts = c->d_tci + 1;
  c->tc_syn.err = c->tc_ana.err = c->d_err;
  c->nsyn = src->nsyn;
  c->nana = src->nana;
  c->tiles_syn_h = src->tiles_syn_h;
  c->tiles_ana_h = src->tiles_ana_h;
  c->tiles_version = src->tiles_version;
}

void destroy_clone(fnl_shells* c) {
  if (c) free_shells(c);
}

void release_shells(fnl_shells* sh) {
  if (sh) free_shells(sh);
}

namespace {

void launch_tc(const fnl_shells* sh, const TcArgs& base, int mode, double* alm_out, cudaStream_t st,
               bool store_f32 = false) {
  TcArgs a = base;
  a.mode = mode;
  a.alm_out = alm_out;
  a.store_f32 = store_f32 ? 1 : 0;
  launch_tc_gemm(a, sh->sms_gemm ? sh->sms_gemm : sh->sms, st);
}

}  // namespace

void launch_synthesis_gemm(const fnl_shells* sh, cudaStream_t st) {
  if (sh->nterms) launch_tc(sh, sh->tc_syn, TC_SYNTH, nullptr, st);
  else launch_synth_gemm(sh, st);
}
}  // namespace fnl

using namespace fnl;

extern "C" {

const char* fnl_version(void) { return "libfnl 0.1 (sm_103a)"; }

const char* fnl_last_error(void) { return g_last_error.c_str(); }

fnl_status fnl_gauss_legendre(int n, double* x, double* w) {
  return guard([&] {
    FNL_REQUIRE(n >= 1 && n <= 100000, "n must be in [1, 100000]");
    FNL_REQUIRE(x && w, "x and w must not be NULL");
    gauss_legendre(n, x, w);
  });
}

fnl_status fnl_covariance(int lmax, int nr, const double* r, double A, double ns, double kmin, double kmax, int nk,
                          double* C) {
  return guard([&] {
    FNL_REQUIRE(lmax >= 0 && lmax <= 4096 && nr >= 1 && nr <= 4096, "bad lmax or nr");
    FNL_REQUIRE(r && C, "r and C must not be NULL");
    FNL_REQUIRE(nk >= 2 && kmin > 0 && kmax > kmin, "need nk >= 2 and 0 < kmin < kmax");
    for (int i = 0; i < nr; ++i) FNL_REQUIRE(r[i] > 0, "r_i must be > 0");
    covariance(lmax, nr, r, A, ns, kmin, kmax, nk, C);
  });
}

fnl_status fnl_cholesky_filters(int lmax, int nr, const double* C, double jitter_rel, double* K) {
  return guard([&] {
    FNL_REQUIRE(lmax >= 0 && nr >= 1 && C && K, "bad arguments");
    cholesky_filters(lmax, nr, C, jitter_rel, K);
  });
}

fnl_status fnl_make_shells(const fnl_shell_desc* d, int device, fnl_shells** out) {
  fnl_shells* sh = nullptr;
  fnl_status st = guard([&] {
    FNL_REQUIRE(out, "out must not be NULL");
    *out = nullptr;
    sh = make_shells_core(d, device, false);
    *out = sh;
  });
  return st;
}

fnl_status fnl_make_shells_shard(const fnl_shell_desc* d, int j0, int j1, int device, fnl_shells** out) {
  return guard([&] {
    FNL_REQUIRE(out, "out must not be NULL");
    *out = nullptr;
    FNL_REQUIRE(d, "desc is NULL");
    FNL_REQUIRE(j0 >= 0 && j0 < j1 && j1 <= d->nr, "the shard must be a range 0 <= j0 < j1 <= nr");
    *out = make_shells_core(d, device, false, 0, j0, j1);
  });
}

fnl_status fnl_shells_shard(const fnl_shells* sh, int* j0, int* nr, int* nr_total) {
  return guard([&] {
    check_shells(sh);
    if (j0) *j0 = sh->j0;
    if (nr) *nr = sh->nr;
    if (nr_total) *nr_total = sh->nr_total;
  });
}

fnl_status fnl_make_shells_healpix(const fnl_shell_desc* d, int nside, int device, fnl_shells** out) {
  return guard([&] {
    FNL_REQUIRE(out, "out must not be NULL");
    *out = nullptr;
    FNL_REQUIRE(nside >= 1, "nside must be >= 1");
    *out = make_shells_core(d, device, false, nside);
  });
}

}  // extern "C"

namespace fnl {

fnl_shells* make_shells_core(const fnl_shell_desc* d_in, int device, bool synth_only, int nside, int sj0, int sj1) {
  fnl_shells* sh = nullptr;
  try {
    FNL_REQUIRE(d_in, "desc is NULL");
    fnl_shell_desc dd = *d_in;
    if (nside) {
      FNL_REQUIRE(nside >= 1 && nside <= 4096 && (nside & (nside - 1)) == 0, "nside must be a power of two <= 4096");
      FNL_REQUIRE(dd.prec == FNL_FP64 || dd.prec == FNL_FP32, "the HEALPix grid runs in the FNL_FP64 and FNL_FP32 forms");
      dd.ntheta = 4 * nside - 1;
      dd.nphi = 4 * nside;
    }
    const fnl_shell_desc* d = &dd;
    const int nr_full = d->nr;
    const bool shard = sj1 >= 0;
    if (shard) {
      // validate the configuration as a whole (its nr is the full shell count), then the range
      FNL_REQUIRE(!synth_only && !nside, "shell shards are made on the Gauss-Legendre grid");
      FNL_REQUIRE(d->nr >= 1, "nr must be >= 1");
      FNL_REQUIRE(sj0 >= 0 && sj0 < sj1 && sj1 <= d->nr, "the shard must be a range 0 <= j0 < j1 <= nr");
      dd.nr = sj1 - sj0;  // the checks of validate_desc on the shard's own shell count
      validate_desc(d, false, false);
      dd.nr = nr_full;
    } else {
      validate_desc(d, synth_only, nside > 0);
      sj0 = 0;
      sj1 = nr_full;
    }
    const bool mixed = (d->prec == FNL_BF16X2 || d->prec == FNL_BF16X3);
    int ndev = 0;
    FNL_CUDA(cudaGetDeviceCount(&ndev));
    FNL_REQUIRE(device >= 0 && device < ndev, "no such CUDA device");
    DeviceScope scope(device);
    if (mixed) {
      int major = 0, minor = 0;
      FNL_CUDA(cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, device));
      FNL_CUDA(cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, device));
      if (major != 10 || minor != 3)
        throw Error(FNL_EUNSUPPORTED, "the tensor-core forms are built for sm_103a only");
    }
    sh = new fnl_shells;
    sh->device = device;
    // nr: the object's shells (j0 .. j0 + nr - 1 of the configuration); ncol: the noise shells
    // their rows of K_l reach
    const int L = d->lmax, j0 = sj0, nr = sj1 - sj0, ncol = sj1;
    sh->lmax = L;
    sh->nr = nr;
    sh->j0 = j0;
    sh->nr_total = nr_full;
    sh->ntheta = d->ntheta;
    sh->nphi = d->nphi;
    sh->prec = d->prec;
    sh->npairs = (d->ntheta + 1) / 2;
    sh->C = 2 * nr;
    sh->nalm = n_alm(L);
    sh->real_is_double = (d->prec == FNL_FP64);
    sh->nterms = d->prec == FNL_BF16X2 ? 2 : d->prec == FNL_BF16X3 ? 3 : 0;
    {
      sh->tc_split = 1;
    }
    FNL_CUDA(cudaDeviceGetAttribute(&sh->sms, cudaDevAttrMultiProcessorCount, device));
    const int np = sh->npairs, C = sh->C;
    const size_t ts = sh->real_is_double ? sizeof(double) : sizeof(float);

    // ---- problem geometry
    const int nmp = 2 * (L + 1);
    sh->K.resize(nmp);
    sh->KP.resize(nmp);
    sh->row0.resize(nmp + 1);
    sh->lam0.resize(nmp + 1);
    int64_t rows = 0, lams = 0;
    for (int mp = 0; mp < nmp; ++mp) {
      const int k = k_of(L, mp / 2, mp % 2);
      sh->K[mp] = k;
      sh->KP[mp] = round_up(k, 16);
      sh->row0[mp] = rows;
      sh->lam0[mp] = lams;
      rows += sh->KP[mp];
      lams += (int64_t)np * sh->KP[mp];
    }
    sh->row0[nmp] = rows;
    sh->lam0[nmp] = lams;
    sh->rows_total = rows;
    sh->lam_total = lams;
    sh->row32.resize(nmp + 1);
    int64_t r32 = 0;
    for (int mp = 0; mp < nmp; ++mp) {
      sh->row32[mp] = r32;
      r32 += round_up(sh->K[mp], 32);
    }
    sh->row32[nmp] = r32;
    sh->Cpad = round_up(C, 128);
    sh->npj = round_up(np, 32);

    // ---- ring grid (northern half): Gauss-Legendre nodes and weights, or the HEALPix rings with
    // the equal-area rule's weight 2 n_j / N_pix per ring (so that (2 pi / n_j) w_j = 4 pi / N_pix)
    sh->nside = nside;
    if (nside) {
      std::vector<double> z, phi0;
      std::vector<int> n;
      healpix_rings(nside, z, n, phi0);
      const double npix = 12.0 * nside * nside;
      sh->x.assign(z.begin(), z.begin() + np);
      sh->wgl.resize(np);
      for (int j = 0; j < np; ++j) sh->wgl[j] = 2.0 * n[j] / npix;
    } else {
      std::vector<double> xg(d->ntheta), wg(d->ntheta);
      gauss_legendre(d->ntheta, xg.data(), wg.data());
      sh->x.assign(xg.begin(), xg.begin() + np);
      sh->wgl.assign(wg.begin(), wg.begin() + np);
    }

    // ---- filters K_l (Eq. 9) of the whole configuration, then the object's rows of them
    const size_t kk = synth_only ? 0 : (size_t)(L + 1) * nr_full * nr_full;
    std::vector<double> Kfull(kk);
    if (synth_only) {
      // a synthesis-only object (internal): no filters, mu, q or v
    } else if (d->K) {
      for (int l = 0; l <= L; ++l)
        for (int i = 0; i < nr_full; ++i)
          for (int j = 0; j < nr_full; ++j)
            Kfull[((size_t)l * nr_full + i) * nr_full + j] = (j <= i) ? d->K[((size_t)l * nr_full + i) * nr_full + j] : 0.0;
    } else {
      std::vector<double> Cv(kk);
      covariance(L, nr_full, d->r, d->A, d->ns, d->kmin, d->kmax, d->nk, Cv.data());
      cholesky_filters(L, nr_full, Cv.data(), d->jitter_rel, Kfull.data());
    }
    for (size_t i = 0; i < kk; ++i) FNL_REQUIRE(std::isfinite(Kfull[i]), "filters contain non-finite values");
    // Kf[l][i][j] = K_l[j0 + i][j], j < ncol: the rows the object computes (all of K_l when whole)
    std::vector<double> Kf(synth_only ? 0 : (size_t)(L + 1) * nr * ncol);
    for (int l = 0; l <= (synth_only ? -1 : L); ++l)
      for (int i = 0; i < nr; ++i)
        for (int j = 0; j < ncol; ++j)
          Kf[((size_t)l * nr + i) * ncol + j] = Kfull[((size_t)l * nr_full + j0 + i) * nr_full + j];

    // ---- mu (Eq. 2), q^X and v^X (Eq. 5) of the object's shells
    sh->mu.assign(nr, 0.0);
    if (synth_only) {
    } else if (d->mu) {
      for (int i = 0; i < nr; ++i) sh->mu[i] = d->mu[j0 + i];
    } else {
      for (int l = 0; l <= L; ++l)
        for (int i = 0; i < nr; ++i) {
          double s = 0.0;
          for (int j = 0; j <= j0 + i; ++j) s += Kf[((size_t)l * nr + i) * ncol + j] * Kf[((size_t)l * nr + i) * ncol + j];
          sh->mu[i] += (2.0 * l + 1.0) / (4.0 * M_PI) * s;
        }
    }
    std::vector<double> qT((size_t)(L + 1) * nr), qE((size_t)(L + 1) * nr);
    std::vector<double> vT((size_t)(L + 1) * ncol, 0.0), vE((size_t)(L + 1) * ncol, 0.0);
    for (int l = 0; l <= L; ++l)
      for (int i = 0; i < nr; ++i) {
        const int g = j0 + i;
        const double f = d->w[g] * d->r[g] * d->r[g];
        qT[(size_t)l * nr + i] = f * d->alphaT[(size_t)l * nr_full + g];
        qE[(size_t)l * nr + i] = f * d->alphaE[(size_t)l * nr_full + g];
      }
    // v^X_l[j] = sum over the object's rows i of K_l[j0 + i][j] q^X_l[i]: a^X_L = v^X . n is then
    // the quadrature of the object's shells of Phi_L (Eq. 5), whatever shards it is split into
    for (int l = 0; l <= (synth_only ? -1 : L); ++l)
      for (int i = 0; i < nr; ++i)
        for (int j = 0; j <= j0 + i; ++j) {
          const double k = Kf[((size_t)l * nr + i) * ncol + j];
          vT[(size_t)l * ncol + j] += k * qT[(size_t)l * nr + i];
          vE[(size_t)l * ncol + j] += k * qE[(size_t)l * nr + i];
        }

    // ---- FFT plan and twiddles e^{-2 pi i k / nphi}
    sh->fft = make_fft_plan(d->nphi);
    std::vector<double> tw(2 * (size_t)d->nphi);
    for (int k = 0; k < d->nphi; ++k) {
      const double a = 2.0 * M_PI * (double)k / (double)d->nphi;
      tw[2 * k] = std::cos(a);
      tw[2 * k + 1] = -std::sin(a);
    }

    // ---- SIMT tile lists: synthesis (rows = ring pairs), analysis (rows = degrees)
    std::vector<Tile> ts_syn, ts_ana;
    const int ctiles = (C + kSimtBN - 1) / kSimtBN, bm = sh->real_is_double ? kSimtBM64 : kSimtBM;
    for (int mp = 0; mp < nmp; ++mp) {
      if (sh->K[mp] == 0) continue;
      for (int rt = 0; rt < (np + bm - 1) / bm; ++rt)
        for (int ct = 0; ct < ctiles; ++ct) ts_syn.push_back({mp, rt, ct, 0});
      for (int rt = 0; rt < (sh->K[mp] + bm - 1) / bm; ++rt)
        for (int ct = 0; ct < ctiles; ++ct) ts_ana.push_back({mp, rt, ct, 0});
    }
    sh->n_tiles_syn = (int)ts_syn.size();
    sh->n_tiles_ana = (int)ts_ana.size();

    // ---- device side
    sh->d_K = upload(sh, sh->K);
    sh->d_row0 = upload(sh, sh->row0);
    sh->d_lam0 = upload(sh, sh->lam0);
    sh->d_x = upload(sh, sh->x);
    sh->d_wgl = upload(sh, sh->wgl);
    sh->d_vT = upload(sh, vT);
    sh->d_vE = upload(sh, vE);
    sh->d_qT = upload(sh, qT);
    sh->d_qE = upload(sh, qE);
    sh->d_qT32 = upload(sh, std::vector<float>(qT.begin(), qT.end()));
    sh->d_qE32 = upload(sh, std::vector<float>(qE.begin(), qE.end()));
    sh->d_mu = upload(sh, sh->mu);
    sh->d_tiles_syn = upload(sh, ts_syn);
    sh->d_tiles_ana = upload(sh, ts_ana);
    // per-pass twiddles of the in-place ring FFT: the flat table's entry r k N / (Ns R)
    std::vector<double> twp(2 * (size_t)std::max(sh->fft.ttotal, 1));
    {
      int ns = 1;
      for (int pi = 0; pi < sh->fft.nrad; ++pi) {
        const int R = sh->fft.rad[pi], stride = d->nphi / (ns * R);
        for (int r = 1; r < R; ++r)
          for (int k = 0; k < ns; ++k) {
            const size_t o = (size_t)sh->fft.toff[pi] + (size_t)(r - 1) * ns + k;
            const int e = r * k * stride;
            twp[2 * o] = tw[2 * e];
            twp[2 * o + 1] = tw[2 * e + 1];
          }
        ns *= R;
      }
    }
    if (sh->real_is_double) {
      sh->d_Kf = upload(sh, Kf);
      sh->d_tw = upload(sh, tw);
      sh->d_twp = upload(sh, twp);
    } else {
      std::vector<float> kf(Kf.begin(), Kf.end()), twf(tw.begin(), tw.end()), twpf(twp.begin(), twp.end());
      sh->d_Kf = upload(sh, kf);
      if (mixed && !synth_only) {
        // the BF16 terms of K_l and their tensor map for the tensor-core filter
        build_filter_terms(sh, Kf);
      }
      sh->d_tw = upload(sh, twf);
      sh->d_twp = upload(sh, twpf);
    }
    sh->d_aL = dalloc<double>(sh, 4 * (size_t)sh->nalm);
    sh->d_aNL = dalloc<double>(sh, 4 * (size_t)sh->nalm);
    sh->d_aOut = dalloc<double>(sh, 4 * (size_t)sh->nalm);
    if (!mixed) {
      sh->d_lam = dalloc<unsigned char>(sh, ts * (size_t)sh->lam_total);
      sh->d_phi = dalloc<unsigned char>(sh, ts * (size_t)sh->rows_total * C);
      const size_t fg = ts * (size_t)nmp * np * C;
      sh->d_F = dalloc<unsigned char>(sh, fg);
      sh->d_G = dalloc<unsigned char>(sh, fg);
      FNL_CUDA(cudaMemset(sh->d_phi, 0, ts * (size_t)sh->rows_total * C));
      FNL_CUDA(cudaMemset(sh->d_F, 0, fg));
      FNL_CUDA(cudaMemset(sh->d_G, 0, fg));
      build_lambda_tables(sh, 0);
      // with jmin known, the SIMT tile lists leave out the polar ring pairs of each order where
      // every |lambda_lm| is negligible: synthesis row tiles wholly below jmin write zeros without
      // a k step, and the analysis skips its 16-ring-pair k steps below jmin
      {
        std::vector<Tile> ts, ta;
        const int ctiles = (C + kSimtBN - 1) / kSimtBN, bm = sh->real_is_double ? kSimtBM64 : kSimtBM;
        for (int mp = 0; mp < nmp; ++mp) {
          if (sh->K[mp] == 0) continue;
          const int jz = sh->jmin[mp / 2];
          const int kp = (sh->K[mp] + 15) / 16 * 16;
          for (int rt = 0; rt < (np + bm - 1) / bm; ++rt)  // zero tiles still write their zeros:
            for (int ct = 0; ct < ctiles; ++ct)           // the adjoint's synthesis writes into G
              ts.push_back({mp, rt, ct, (rt + 1) * bm <= jz ? kp : 0});
          for (int rt = 0; rt < (sh->K[mp] + bm - 1) / bm; ++rt)
            for (int ct = 0; ct < ctiles; ++ct) ta.push_back({mp, rt, ct, jz / 16 * 16});
        }
        FNL_REQUIRE(ts.size() <= (size_t)sh->n_tiles_syn && ta.size() <= (size_t)sh->n_tiles_ana, "tile lists");
        FNL_CUDA(cudaMemcpy(sh->d_tiles_syn, ts.data(), sizeof(Tile) * ts.size(), cudaMemcpyHostToDevice));
        FNL_CUDA(cudaMemcpy(sh->d_tiles_ana, ta.data(), sizeof(Tile) * ta.size(), cudaMemcpyHostToDevice));
        sh->n_tiles_syn = (int)ts.size();
        sh->n_tiles_ana = (int)ta.size();
      }
      if (nside) setup_healpix(sh);
    } else {
      setup_mixed(sh, qT, qE);
      if (!synth_only) {
        // the adjoint's second spectrum buffer and its per-shell analysis output
        sh->d_F2 = dalloc<float>(sh, (size_t)nmp * np * sh->Cpad);
        sh->d_adjA = dalloc<float>(sh, 2 * (size_t)sh->nalm * nr);
        sh->tmF2 = f_tensor_map(sh, sh->d_F2);
        FNL_CUDA(cudaMemset(sh->d_F2, 0, sizeof(float) * (size_t)nmp * np * sh->Cpad));
      }
    }
    FNL_CUDA(cudaDeviceSynchronize());
    auto hs = std::make_shared<HostSetup>();
    hs->K = std::move(Kf);
    hs->r.assign(d->r + j0, d->r + j0 + nr);
    hs->w.assign(d->w + j0, d->w + j0 + nr);
    hs->alphaT.resize((size_t)(L + 1) * nr);
    hs->alphaE.resize((size_t)(L + 1) * nr);
    for (int l = 0; l <= L; ++l)
      for (int i = 0; i < nr; ++i) {
        hs->alphaT[(size_t)l * nr + i] = d->alphaT[(size_t)l * nr_full + j0 + i];
        hs->alphaE[(size_t)l * nr + i] = d->alphaE[(size_t)l * nr_full + j0 + i];
      }
    hs->vT = std::move(vT);
    hs->vE = std::move(vE);
    sh->host = hs;
    sh->synth_only = synth_only;
  } catch (...) {
    if (sh) free_shells(sh);
    throw;
  }
  return sh;
}

}  // namespace fnl

extern "C" {

void fnl_shells_destroy(fnl_shells* sh) {
  if (!sh) return;
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(sh->device);
  cudaDeviceSynchronize();
  free_shells(sh);
  if (prev >= 0) cudaSetDevice(prev);
}

fnl_status fnl_shells_info(const fnl_shells* sh, int* lmax, int* nr, int* ntheta, int* nphi, int* prec,
                           size_t* device_bytes) {
  return guard([&] {
    check_shells(sh);
    if (lmax) *lmax = sh->lmax;
    if (nr) *nr = sh->nr;
    if (ntheta) *ntheta = sh->ntheta;
    if (nphi) *nphi = sh->nphi;
    if (prec) *prec = sh->prec;
    if (device_bytes) *device_bytes = sh->device_bytes;
  });
}

fnl_status fnl_shells_mu(const fnl_shells* sh, double* mu_out) {
  return guard([&] {
    check_shells(sh);
    FNL_REQUIRE(mu_out, "mu_out must not be NULL");
    for (int i = 0; i < sh->nr; ++i) mu_out[i] = sh->mu[i];
  });
}

fnl_status fnl_filter(const fnl_shells* sh, uint64_t seed, uint64_t realisation, const double* noise, double* phiL,
                      void* stream) {
  return guard([&] {
    check_shells(sh);
    DeviceScope scope(sh->device);
    check_dev_ptr(noise, "noise", true);
    check_dev_ptr(phiL, "phiL", false);
    cudaStream_t st = (cudaStream_t)stream;
    if (sh->nterms)
      launch_filter_mixed(sh, seed, realisation, noise, sh->d_aL, sh->d_aL + 2 * sh->nalm, phiL, nullptr, st);
    else launch_filter(sh, seed, realisation, noise, sh->d_aL, sh->d_aL + 2 * sh->nalm, phiL, st);
  });
}

fnl_status fnl_synth(const fnl_shells* sh, const double* alm, double* maps, void* stream) {
  return guard([&] {
    check_shells(sh);
    DeviceScope scope(sh->device);
    check_dev_ptr(alm, "alm", false);
    check_dev_ptr(maps, "maps", false);
    cudaStream_t st = (cudaStream_t)stream;
    if (sh->nterms) {
      launch_alm_to_terms(sh, alm, st);
      launch_tc(sh, sh->tc_syn, TC_SYNTH, nullptr, st);
    } else {
      launch_alm_to_phi(sh, alm, st);
      launch_synth_gemm(sh, st);
    }
    launch_ring_fft(sh, FFT_SYNTH_MAP, nullptr, maps, st);
  });
}

fnl_status fnl_shells_set_sm_limits(fnl_shells* sh, int gemm_sms, int ring_sms) {
  return guard([&] {
    check_shells(sh);
    FNL_REQUIRE(gemm_sms >= 0 && gemm_sms <= sh->sms && ring_sms >= 0 && ring_sms <= sh->sms,
                "SM limits must be in [0, the device's SM count]");
    sh->sms_gemm = gemm_sms;
    sh->sms_ring = ring_sms;
  });
}

fnl_status fnl_maps_prepare(fnl_shells* sh) {
  return guard([&] {
    check_shells(sh);
    if (sh->nside) throw Error(FNL_EUNSUPPORTED, "the Stokes maps run on the Gauss-Legendre grid");
    FNL_REQUIRE(!sh->owner, "fnl_maps_prepare: not on a scratch clone");
    DeviceScope scope(sh->device);
    maps_prepare(sh);
  });
}

fnl_status fnl_maps(const fnl_shells* sh, const double* aT, const double* aE, const double* aB, double* maps,
                    void* stream) {
  return guard([&] {
    check_shells(sh);
    FNL_REQUIRE(sh->maps_ready, "fnl_maps: call fnl_maps_prepare first");
    DeviceScope scope(sh->device);
    check_dev_ptr(aT, "aT", false);
    check_dev_ptr(aE, "aE", false);
    check_dev_ptr(aB, "aB", true);
    check_dev_ptr(maps, "maps", false);
    launch_maps(sh, aT, aE, aB, maps, (cudaStream_t)stream);
  });
}

fnl_status fnl_analyse(const fnl_shells* sh, const double* maps, double* alm, void* stream) {
  return guard([&] {
    check_shells(sh);
    DeviceScope scope(sh->device);
    check_dev_ptr(maps, "maps", false);
    check_dev_ptr(alm, "alm", false);
    cudaStream_t st = (cudaStream_t)stream;
    launch_ring_fft(sh, FFT_ANALYSE_MAP, maps, nullptr, st);
    if (sh->nterms) {
      launch_tc(sh, sh->tc_ana, TC_ANA_STORE, alm, st);
    } else {
      launch_analysis_gemm(sh, st);
      launch_phi_to_alm(sh, alm, st);
    }
  });
}

fnl_status fnl_square(const fnl_shells* sh, const double* phiL, double* phiNL, void* stream) {
  return guard([&] {
    check_shells(sh);
    DeviceScope scope(sh->device);
    check_dev_ptr(phiL, "phiL", false);
    check_dev_ptr(phiNL, "phiNL", false);
    cudaStream_t st = (cudaStream_t)stream;
    if (sh->nterms) {
      launch_alm_to_terms(sh, phiL, st);
      launch_tc(sh, sh->tc_syn, TC_SYNTH, nullptr, st);
      launch_ring_fft(sh, FFT_SQUARE, nullptr, nullptr, st);
      launch_tc(sh, sh->tc_ana, TC_ANA_STORE, phiNL, st);
    } else {
      launch_alm_to_phi(sh, phiL, st);
      launch_synth_gemm(sh, st);
      launch_ring_fft(sh, FFT_SQUARE, nullptr, nullptr, st);
      launch_analysis_gemm(sh, st);
      launch_phi_to_alm(sh, phiNL, st);
    }
  });
}

fnl_status fnl_accumulate(const fnl_shells* sh, const double* phiL, const double* phiNL, double fnl, double* aT,
                          double* aE, double* aLT, double* aLE, double* aNLT, double* aNLE, void* stream) {
  return guard([&] {
    check_shells(sh);
    DeviceScope scope(sh->device);
    check_dev_ptr(phiL, "phiL", true);
    check_dev_ptr(phiNL, "phiNL", true);
    for (auto pr : {std::make_pair((const void*)aT, "aT"), std::make_pair((const void*)aE, "aE"),
                    std::make_pair((const void*)aLT, "aLT"), std::make_pair((const void*)aLE, "aLE"),
                    std::make_pair((const void*)aNLT, "aNLT"), std::make_pair((const void*)aNLE, "aNLE")})
      check_dev_ptr(pr.first, pr.second, true);
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n2 = 2 * sh->nalm;
    double* lT = aLT ? aLT : sh->d_aL;
    double* lE = aLE ? aLE : sh->d_aL + n2;
    double* nT = aNLT ? aNLT : sh->d_aNL;
    double* nE = aNLE ? aNLE : sh->d_aNL + n2;
    if (phiL) launch_quadrature(sh, phiL, 0, 0.0, nullptr, nullptr, nullptr, nullptr, lT, lE, 0, st);
    else {
      FNL_CUDA(cudaMemsetAsync(lT, 0, sizeof(double) * n2, st));
      FNL_CUDA(cudaMemsetAsync(lE, 0, sizeof(double) * n2, st));
    }
    if (phiNL) launch_quadrature(sh, phiNL, 0, fnl, lT, lE, aT, aE, nT, nE, 0, st);
    else {
      FNL_CUDA(cudaMemsetAsync(nT, 0, sizeof(double) * n2, st));
      FNL_CUDA(cudaMemsetAsync(nE, 0, sizeof(double) * n2, st));
      launch_combine(sh, fnl, lT, lE, nT, nE, aT, aE, st);
    }
  });
}

}  // extern "C"

namespace fnl {

// Steps (i)-(v) for one realisation, outputs in device memory (NULL -> scratch).
void run_generate(const fnl_shells* sh, uint64_t seed, uint64_t realisation, double fnl, const double* noise,
                  double* aT, double* aE, double* aLT, double* aLE, double* aNLT, double* aNLE, cudaStream_t st,
                  bool mark_events) {
  const int64_t n2 = 2 * sh->nalm;
  double* lT = aLT ? aLT : sh->d_aL;
  double* lE = aLE ? aLE : sh->d_aL + n2;
  double* nT = aNLT ? aNLT : sh->d_aNL;
  double* nE = aNLE ? aNLE : sh->d_aNL + n2;
  fnl_shells* msh = const_cast<fnl_shells*>(sh);
  cudaEvent_t* ev = nullptr;
  if (sh->ring_slots && mark_events) {
    ev = msh->ring.data() + (size_t)sh->ring_head * (FNL_NSTAGES + 1);
    msh->ring_head = (sh->ring_head + 1) % sh->ring_slots;
    msh->ring_count = std::min(sh->ring_count + 1, sh->ring_slots);
  }
  auto mark = [&](int i) {
    if (ev) FNL_CUDA(cudaEventRecord(ev[i], st));
  };
  mark(0);
  if (sh->nterms) {
    launch_filter_mixed(sh, seed, realisation, noise, lT, lE, nullptr, sh->d_psum, st);  // (i)
    mark(1);
    launch_tc(sh, sh->tc_syn, TC_SYNTH, nullptr, st);                         // (ii) Legendre
    mark(2);
    launch_ring_fft(sh, FFT_SQUARE, nullptr, nullptr, st);                    // (ii) DFT, (iii), (iv) DFT
    mark(3);
    launch_tc(sh, sh->tc_ana, TC_ANA_QUAD, nullptr, st);                      // (iv) Legendre + (v)
    mark(4);
    launch_combine_mixed(sh, fnl, lT, lE, nT, nE, aT, aE, sh->d_psum, st);   // (v), Eq. 3
  } else {
    launch_filter(sh, seed, realisation, noise, lT, lE, nullptr, st);        // (i)
    mark(1);
    launch_synth_gemm(sh, st);                                              // (ii) Legendre
    mark(2);
    launch_ring_fft(sh, FFT_SQUARE, nullptr, nullptr, st);                  // (ii) DFT, (iii), (iv) DFT
    mark(3);
    launch_analysis_gemm(sh, st);                                           // (iv) Legendre
    mark(4);
    launch_quadrature(sh, nullptr, 1, fnl, lT, lE, aT, aE, nT, nE, 0, st);  // (v)
  }
  mark(5);
}

}  // namespace fnl

extern "C" {

fnl_status fnl_generate(const fnl_shells* sh, uint64_t seed, uint64_t realisation, double fnl, const double* noise,
                        double* aT, double* aE, double* aLT, double* aLE, double* aNLT, double* aNLE, void* stream) {
  return guard([&] {
    check_shells(sh);
    DeviceScope scope(sh->device);
    check_dev_ptr(noise, "noise", true);
    for (auto pr : {std::make_pair((const void*)aT, "aT"), std::make_pair((const void*)aE, "aE"),
                    std::make_pair((const void*)aLT, "aLT"), std::make_pair((const void*)aLE, "aLE"),
                    std::make_pair((const void*)aNLT, "aNLT"), std::make_pair((const void*)aNLE, "aNLE")})
      check_dev_ptr(pr.first, pr.second, true);
    run_generate(sh, seed, realisation, fnl, noise, aT, aE, aLT, aLE, aNLT, aNLE, (cudaStream_t)stream);
  });
}

fnl_status fnl_generate_backward(const fnl_shells* sh, uint64_t seed, uint64_t realisation, double fnl,
                                 const double* noise, const double* gT, const double* gE, const double* aNLT,
                                 const double* aNLE, double* grad_noise, double* grad_fnl, void* stream) {
  return guard([&] {
    check_shells(sh);
    DeviceScope scope(sh->device);
    if (sh->nside) throw Error(FNL_EUNSUPPORTED, "fnl_generate_backward runs on the Gauss-Legendre grid");
    if (sh->nr != sh->nr_total)
      throw Error(FNL_EUNSUPPORTED, "fnl_generate_backward needs a whole configuration, not a shell shard");
    if (sh->nterms && (!sh->d_F2 || sh->owner))
      throw Error(FNL_EUNSUPPORTED, "fnl_generate_backward needs a shells object made by fnl_make_shells");
    check_dev_ptr(noise, "noise", true);
    check_dev_ptr(gT, "gT", true);
    check_dev_ptr(gE, "gE", true);
    check_dev_ptr(aNLT, "aNLT", true);
    check_dev_ptr(aNLE, "aNLE", true);
    check_dev_ptr(grad_noise, "grad_noise", true);
    if (grad_fnl) {
      if (((uintptr_t)grad_fnl) % 8 != 0) throw Error(FNL_EINVAL, "grad_fnl must be 8-byte aligned");
      cudaPointerAttributes attr;
      if (cudaPointerGetAttributes(&attr, grad_fnl) != cudaSuccess ||
          (attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged)) {
        cudaGetLastError();
        throw Error(FNL_EINVAL, "grad_fnl must be device memory");
      }
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n2 = 2 * sh->nalm;
    if (grad_fnl) {
      if (!aNLT || !aNLE) {
        // a^X_NL of the forward call, recomputed into the object's scratch
        run_generate(sh, seed, realisation, fnl, noise, nullptr, nullptr, nullptr, nullptr, sh->d_aNL,
                     sh->d_aNL + n2, st);
        aNLT = sh->d_aNL;
        aNLE = sh->d_aNL + n2;
      }
      launch_dot_fnl(sh, gT, gE, aNLT, aNLE, grad_fnl, st);
    }
    if (!grad_noise) return;
    if (sh->nterms) {
      // the same chain on the tensor cores: both syntheses and the analysis are tcgen05 GEMMs
      launch_filter_mixed(sh, seed, realisation, noise, sh->d_aL, sh->d_aL + n2, nullptr, nullptr, st);  // Phi_L
      launch_tc(sh, sh->tc_syn, TC_SYNTH, nullptr, st);                                   // F of f
      launch_adjoint_source(sh, fnl, gT, gE, st);                                        // H~ as BF16 terms
      TcArgs syn2 = sh->tc_syn;
      syn2.one.F = (float*)sh->d_F2;
      syn2.one.tmF = sh->tmF2;
      launch_tc(sh, syn2, TC_SYNTH, nullptr, st);                                         // F of s
      launch_ring_product(sh, st);                                                        // G = DFT(2 f s)
      launch_tc(sh, sh->tc_ana, TC_ANA_STORE, (double*)sh->d_adjA, st, true);            // analysis(2 f s), FP32
      launch_adjoint_filter(sh, gT, gE, grad_noise, st);                                  // K^T (c_m rows + q g)
      return;
    }
    launch_filter(sh, seed, realisation, noise, sh->d_aL, sh->d_aL + n2, nullptr, st);  // Phi_L rows
    launch_synth_gemm(sh, st);                                                          // F of f
    launch_adjoint_source(sh, fnl, gT, gE, st);                                         // rows of H~
    launch_synth_gemm_to(sh, sh->d_G, st);                                              // F of s, in G
    launch_ring_product(sh, st);                                                        // G = DFT(2 f s)
    launch_analysis_gemm(sh, st);                                                       // rows of analysis(2 f s)
    launch_adjoint_filter(sh, gT, gE, grad_noise, st);                                  // K^T (c_m rows + q g)
  });
}

fnl_status fnl_generate_host(const fnl_shells* sh, uint64_t seed, uint64_t realisation, double fnl, double* aT,
                             double* aE, double* aNLT, double* aNLE, void* stream) {
  return guard([&] {
    check_shells(sh);
    DeviceScope scope(sh->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n2 = 2 * sh->nalm;
    const size_t bytes = sizeof(double) * (size_t)n2;
    // page-locked host buffers are written by the last kernel itself, through their device
    // mapping (over the chip-to-chip link where the host memory sits); other buffers get a copy
    auto mapped = [](double* h) -> double* {
      if (!h) return nullptr;
      cudaPointerAttributes at{};
      if (cudaPointerGetAttributes(&at, h) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
      }
      return at.type == cudaMemoryTypeHost && at.devicePointer ? (double*)at.devicePointer : nullptr;
    };
    double* mT = mapped(aT);
    double* mE = mapped(aE);
    double* mNT = mapped(aNLT);
    double* mNE = mapped(aNLE);
    double* dT = mT ? mT : sh->d_aOut;
    double* dE = mE ? mE : sh->d_aOut + n2;
    run_generate(sh, seed, realisation, fnl, nullptr, dT, dE, nullptr, nullptr, mNT, mNE, st);
    if (aT && !mT) FNL_CUDA(cudaMemcpyAsync(aT, dT, bytes, cudaMemcpyDeviceToHost, st));
    if (aE && !mE) FNL_CUDA(cudaMemcpyAsync(aE, dE, bytes, cudaMemcpyDeviceToHost, st));
    if (aNLT && !mNT) FNL_CUDA(cudaMemcpyAsync(aNLT, sh->d_aNL, bytes, cudaMemcpyDeviceToHost, st));
    if (aNLE && !mNE) FNL_CUDA(cudaMemcpyAsync(aNLE, sh->d_aNL + n2, bytes, cudaMemcpyDeviceToHost, st));
  });
}

fnl_status fnl_profile_enable(fnl_shells* sh, int slots) {
  return guard([&] {
    check_shells(sh);
    FNL_REQUIRE(slots >= 0 && slots <= 4096, "slots must be in [0, 4096]");
    DeviceScope scope(sh->device);
    FNL_CUDA(cudaDeviceSynchronize());
    for (auto& e : sh->ring)
      if (e) cudaEventDestroy(e);
    sh->ring.assign((size_t)slots * (FNL_NSTAGES + 1), nullptr);
    for (auto& e : sh->ring) FNL_CUDA(cudaEventCreate(&e));
    sh->ring_slots = slots;
    sh->ring_head = 0;
    sh->ring_count = 0;
  });
}

fnl_status fnl_profile_read(fnl_shells* sh, double* ms, int n, int* calls) {
  return guard([&] {
    check_shells(sh);
    FNL_REQUIRE(ms && n >= 1 && n <= FNL_NSTAGES, "need 1 <= n <= FNL_NSTAGES and ms != NULL");
    FNL_REQUIRE(sh->ring_slots > 0, "profiling is off");
    DeviceScope scope(sh->device);
    for (int i = 0; i < n; ++i) ms[i] = 0.0;
    for (int c = 0; c < sh->ring_count; ++c) {
      const int slot = (sh->ring_head - 1 - c + 2 * sh->ring_slots) % sh->ring_slots;
      cudaEvent_t* ev = sh->ring.data() + (size_t)slot * (FNL_NSTAGES + 1);
      FNL_CUDA(cudaEventSynchronize(ev[FNL_NSTAGES]));
      for (int i = 0; i < n; ++i) {
        float t = 0.f;
        FNL_CUDA(cudaEventElapsedTime(&t, ev[i], ev[i + 1]));
        ms[i] += t;
      }
    }
    if (calls) *calls = sh->ring_count;
    sh->ring_count = 0;
  });
}

fnl_status fnl_test_fail_alloc(long n) {
  return guard([&] {
    FNL_REQUIRE(n >= -1, "n must be >= -1");
    g_fail_alloc.store(n);
  });
}

fnl_status fnl_test_wait_expiry(const fnl_shells* sh, unsigned limit, void* stream) {
  return guard([&] {
    check_shells(sh);
    FNL_REQUIRE(sh->d_err, "fnl_test_wait_expiry: a tensor-core object is needed (it owns the error word)");
    FNL_REQUIRE(limit >= 1 && limit <= (1u << 20), "limit must be in [1, 2^20]");
    DeviceScope scope(sh->device);
    launch_wait_probe(sh->d_err, limit, (cudaStream_t)stream);
  });
}

fnl_status fnl_device_status(const fnl_shells* sh) {
  return guard([&] {
    check_shells(sh);
    DeviceScope scope(sh->device);
    FNL_CUDA(cudaDeviceSynchronize());
    if (!sh->d_err) return;
    int e = 0;
    FNL_CUDA(cudaMemcpy(&e, sh->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (e) {
      FNL_CUDA(cudaMemset(sh->d_err, 0, sizeof(int)));
      throw Error(FNL_ETIMEOUT, "a bounded wait in a tensor-core kernel expired (code " + std::to_string(e) + ")");
    }
  });
}

}  // extern "C"
