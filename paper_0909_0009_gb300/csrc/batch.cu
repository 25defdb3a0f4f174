// Batching form: many realisations of uneven l_max and N_r in one captured CUDA graph, and
// the autotuners that pick the tensor-core tile shapes.
//
// A batch holds n instances, each a (shells object, seed, realisation, f_NL) of steps
// (i)-(v) (Sect. 2).  Every instance gets scratch of its own: the first instance of a
// shells object uses the object's, later ones use scratch clones that share its tables.
//
// Multi-instance mode (every instance a whole configuration in a tensor-core form with a
// specialised ring kernel, at most kTcMaxInst of them): each stage after the filter is ONE
// launch over all instances --
//   k_filter_tc + k_psum_reduce     step (i): the tensor-core filter of each instance, the same
//                                   launches as its single call (a persistent kernel per instance)
//   k_tc_gemm<true>, synthesis      step (ii) Legendre: one persistent tile list over all
//                                   instances (instance tensor maps in constant memory)
//   k_ring_square<.., true>         steps (ii)-(iv) ring DFTs and square, one launch per ring
//                                   length present (the kernel is specialised per length)
//   k_tc_gemm<true>, analysis       steps (iv), (v)
//   k_combine_multi                 Eq. 3
// so a batch of n realisations is 2 n + 3 + (ring lengths) launches, captured into one graph
// per call (an update of the instantiated graph) with the call's keys and outputs.  The tile
// shape, the same for every instance of a launch, is picked by timing whole batches
// (fnl_batch_create).
//
// Stream mode (any other batch: SIMT forms, ring lengths without a specialised kernel):
// instances are dealt, largest first (work ~ (l_max + 1)^3 N_r), to up to `nstreams`
// streams; instances that share scratch (repeated SIMT objects) stay on one stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <numeric>
#include <vector>

#include "fnl_internal.cuh"

using fnl::CombineInst;
using fnl::TcArgs;
using fnl::TcInst;
using fnl::TcTile;

struct fnl_batch {
  int device = 0;
  int n = 0;
  std::vector<fnl_shells*> sh;      // per instance: the caller's object
  std::vector<fnl_shells*> run;     // per instance: the object whose scratch it uses
  std::vector<fnl_shells*> clones;  // owned scratch clones
  bool multi = false;
  // stream mode
  std::vector<int> lane;
  std::vector<std::vector<int>> order;
  std::vector<cudaStream_t> streams;  // streams[0] also begins the capture
  std::vector<cudaEvent_t> joins;
  cudaEvent_t fork = nullptr;
  // multi-instance mode
  int syn_w = 0, ana_w = 0;           // tile widths of both GEMM launches
  std::vector<int> versions;          // tile versions of the owners when the arrays were built
  std::vector<void*> dev;             // device arrays (owned)
  void* pinned = nullptr;             // host tensor maps (owned, pinned)
  TcArgs tsyn{}, tana{};
  CUtensorMap* h_maps_syn = nullptr;
  CUtensorMap* h_maps_ana = nullptr;
  struct Ring {
    const fnl_shells* proto;
    void* d_args;
    int* d_item0;
    int ninst, maxL, items;
  };
  std::vector<Ring> rings;
  CombineInst* d_cinst = nullptr;
  int64_t max_nalm = 0;
  cudaGraphExec_t exec = nullptr;
};

namespace fnl {
namespace {

double work_of(const fnl_shells* s) { return (double)(s->lmax + 1) * (s->lmax + 1) * (s->lmax + 1) * s->nr; }

const fnl_shells* owner_of(const fnl_shells* s) { return s->owner ? s->owner : s; }

void free_multi_arrays(fnl_batch* b) {
  for (void* p : b->dev) cudaFree(p);
  b->dev.clear();
  if (b->pinned) cudaFreeHost(b->pinned);
  b->pinned = nullptr;
  b->rings.clear();
}

void free_batch(fnl_batch* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  for (cudaEvent_t e : b->joins)
    if (e) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  for (cudaStream_t s : b->streams)
    if (s) cudaStreamDestroy(s);
  free_multi_arrays(b);
  for (fnl_shells* c : b->clones) destroy_clone(c);
  delete b;
}

template <typename T>
T* upload_vec(fnl_batch* b, const std::vector<T>& v) {
  void* p = nullptr;
  FNL_CUDA(cudaMalloc(&p, sizeof(T) * std::max<size_t>(v.size(), 1)));
  b->dev.push_back(p);
  FNL_CUDA(cudaMemcpy(p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice));
  return (T*)p;
}

// Tile shape `w` on every owner (exact widths), clones refreshed, launch arrays rebuilt.
void build_multi(fnl_batch* b, int syn_w, int ana_w) {
  FNL_CUDA(cudaDeviceSynchronize());
  free_multi_arrays(b);
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  std::vector<const fnl_shells*> owners;
  for (fnl_shells* r : b->run)
    if (std::find(owners.begin(), owners.end(), owner_of(r)) == owners.end()) owners.push_back(owner_of(r));
  for (const fnl_shells* o : owners) configure_tc(const_cast<fnl_shells*>(o), syn_w, ana_w, true);
  for (fnl_shells* c : b->clones) refresh_clone(c, c->owner);
  b->syn_w = syn_w;
  b->ana_w = ana_w;
  b->versions.clear();
  for (fnl_shells* r : b->run) b->versions.push_back(owner_of(r)->tiles_version);
  const int n = b->n;

  // step (v): the instances' combine arguments
  std::vector<CombineInst> ci(n);
  b->max_nalm = 0;
  for (int i = 0; i < n; ++i) {
    const fnl_shells* s = b->run[i];
    const int64_t n2 = 2 * s->nalm;
    ci[i] = CombineInst{s->nalm, s->Cpad / 128, s->nr, (const double2*)s->d_part, s->d_psum, s->d_mu, s->d_qT,
                        s->d_qE, (const double2*)s->d_aL, (const double2*)(s->d_aL + n2), (double2*)s->d_aNL,
                        (double2*)(s->d_aNL + n2)};
    b->max_nalm = std::max(b->max_nalm, s->nalm);
  }
  b->d_cinst = upload_vec(b, ci);

  // Legendre GEMMs: one tile list over all instances, the tiles of one (instance, problem)
  // adjacent, groups largest first; instance maps for the constant table
  FNL_CUDA(cudaMallocHost(&b->pinned, sizeof(CUtensorMap) * 6 * (size_t)n));
  b->h_maps_syn = (CUtensorMap*)b->pinned;
  b->h_maps_ana = b->h_maps_syn + 3 * (size_t)n;
  for (int dir = 0; dir < 2; ++dir) {
    std::vector<TcInst> insts(n);
    // (work, configuration, tiles) of every (instance, problem); equal work is kept together by
    // configuration, so that instances sharing one Legendre table (repeats of an object) read
    // its slabs back to back and find them in L2
    struct Group {
      int64_t work;
      int cfg;
      std::vector<TcTile> tiles;
    };
    std::vector<Group> groups;
    std::vector<const fnl_shells*> cfgs;
    for (int i = 0; i < n; ++i) {
      const fnl_shells* s = b->run[i];
      const fnl_shells* o = owner_of(s);
      const int cfg = (int)(std::find(cfgs.begin(), cfgs.end(), o) - cfgs.begin());
      if (cfg == (int)cfgs.size()) cfgs.push_back(o);
      insts[i] = s->tci[dir];
      CUtensorMap* maps = (dir ? b->h_maps_ana : b->h_maps_syn) + 3 * (size_t)i;
      maps[0] = s->tci[dir].tmA;
      maps[1] = s->tci[dir].tmB;
      maps[2] = s->tci[0].tmF;  // read by the synthesis epilogue only
      const std::vector<TcTile>& tl = dir ? s->tiles_ana_h : s->tiles_syn_h;
      for (size_t k = 0; k < tl.size(); ++k) {
        if (k == 0 || tl[k].mp != tl[k - 1].mp) groups.push_back({0, cfg, {}});
        TcTile t = tl[k];
        t.inst = i;
        groups.back().work += (int64_t)(t.nkb - t.kb0) * t.nsize;
        groups.back().tiles.push_back(t);
      }
    }
    std::stable_sort(groups.begin(), groups.end(), [](const Group& a, const Group& c) {
      return a.work != c.work ? a.work > c.work : a.cfg < c.cfg;
    });
    std::vector<TcTile> tiles;
    for (const auto& g : groups) tiles.insert(tiles.end(), g.tiles.begin(), g.tiles.end());
    TcArgs a = dir ? b->run[0]->tc_ana : b->run[0]->tc_syn;
    a.one = TcInst{};
    a.multi = 1;
    a.insts = upload_vec(b, insts);
    a.tiles = upload_vec(b, tiles);
    a.ntiles = (int)tiles.size();
    a.alm_out = nullptr;
    a.store_f32 = 0;
    a.err = b->run[0]->d_err;
    (dir ? b->tana : b->tsyn) = a;
  }

  // ring kernels: one launch per ring length
  std::map<int, std::vector<int>> by_n;
  for (int i = 0; i < n; ++i) by_n[b->run[i]->nphi].push_back(i);
  const size_t asz = ring_square_args_size();
  for (const auto& kv : by_n) {
    fnl_batch::Ring r{};
    r.proto = b->run[kv.second[0]];
    r.ninst = (int)kv.second.size();
    std::vector<unsigned char> args(asz * r.ninst);
    std::vector<int> item0(1, 0);
    const int G = ring_square_group(r.proto);
    for (int k = 0; k < r.ninst; ++k) {
      const fnl_shells* s = b->run[kv.second[k]];
      ring_square_args(s, args.data() + asz * k);
      item0.push_back(item0.back() + (s->nr / G) * s->npairs);
      r.maxL = std::max(r.maxL, s->lmax);
    }
    r.items = item0.back();
    r.d_args = upload_vec(b, args);
    r.d_item0 = upload_vec(b, item0);
    b->rings.push_back(r);
  }
}

// The launches of one batch call on `st` (no synchronisation; captured by the caller).
void enqueue_multi(fnl_batch* b, const uint64_t* seeds, const uint64_t* reals, const double* fnl, double* const* aT,
                   double* const* aE, cudaStream_t st) {
  MultiOut out{};
  for (int i = 0; i < b->n; ++i) {
    out.fnl[i] = fnl[i];
    out.aT[i] = (double2*)aT[i];
    out.aE[i] = (double2*)aE[i];
  }
  // step (i): the tensor-core filter of each instance (the same launch as its single call)
  for (int i = 0; i < b->n; ++i) {
    const fnl_shells* s = b->run[i];
    launch_filter_mixed(s, seeds[i], reals[i], nullptr, s->d_aL, s->d_aL + 2 * s->nalm, nullptr, s->d_psum, st);
  }
  upload_tc_maps(b->h_maps_syn, b->n, st);
  launch_tc_gemm(b->tsyn, b->run[0]->sms, st);
  for (const fnl_batch::Ring& r : b->rings)
    launch_ring_square_multi(r.proto, r.d_args, r.d_item0, r.ninst, r.maxL, r.items, st);
  upload_tc_maps(b->h_maps_ana, b->n, st);
  launch_tc_gemm(b->tana, b->run[0]->sms, st);
  launch_combine_multi(b->d_cinst, b->max_nalm, b->n, out, st);
}

void enqueue_streams(fnl_batch* b, const uint64_t* seeds, const uint64_t* reals, const double* fnl, double* const* aT,
                     double* const* aE, cudaStream_t cap) {
  FNL_CUDA(cudaEventRecord(b->fork, cap));
  for (size_t l = 1; l < b->streams.size(); ++l) FNL_CUDA(cudaStreamWaitEvent(b->streams[l], b->fork, 0));
  for (size_t l = 0; l < b->streams.size(); ++l) {
    for (int i : b->order[l])
      run_generate(b->run[i], seeds[i], reals[i], fnl[i], nullptr, aT[i], aE[i], nullptr, nullptr, nullptr, nullptr,
                   b->streams[l], false);
    if (l) {
      FNL_CUDA(cudaEventRecord(b->joins[l], b->streams[l]));
      FNL_CUDA(cudaStreamWaitEvent(cap, b->joins[l], 0));
    }
  }
}

// Capture one call into a graph, update or instantiate the batch's executable graph and
// launch it on `stream`.
void run_batch(fnl_batch* b, const uint64_t* seeds, const uint64_t* reals, const double* fnl, double* const* aT,
               double* const* aE, cudaStream_t stream) {
  cudaStream_t cap = b->streams[0];
  cudaGraph_t graph = nullptr;
  FNL_CUDA(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
  try {
    if (b->multi) enqueue_multi(b, seeds, reals, fnl, aT, aE, cap);
    else enqueue_streams(b, seeds, reals, fnl, aT, aE, cap);
  } catch (...) {
    cudaStreamEndCapture(cap, &graph);
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    throw;
  }
  FNL_CUDA(cudaStreamEndCapture(cap, &graph));
  bool ok = false;
  if (b->exec) {
    cudaGraphExecUpdateResultInfo info;
    ok = cudaGraphExecUpdate(b->exec, graph, &info) == cudaSuccess;
    if (!ok) {
      cudaGetLastError();
      cudaGraphExecDestroy(b->exec);
      b->exec = nullptr;
    }
  }
  cudaError_t e = cudaSuccess;
  if (!ok) e = cudaGraphInstantiate(&b->exec, graph, 0);
  cudaGraphDestroy(graph);
  FNL_CUDA(e);
  FNL_CUDA(cudaGraphLaunch(b->exec, stream));
}

// Multi-instance tile shapes tried by fnl_batch_create: whole batches are timed (one
// warm-up, two timed, keys 0 and outputs in the instances' scratch) for each.
void autotune_multi(fnl_batch* b) {
  const int cand[][2] = {{112, 128}, {128, 128}, {96, 128}, {112, 256}};
  std::vector<uint64_t> z(b->n, 0);
  std::vector<double> f(b->n, 1.0);
  std::vector<double*> oT(b->n), oE(b->n);
  for (int i = 0; i < b->n; ++i) {
    oT[i] = b->run[i]->d_aOut;
    oE[i] = b->run[i]->d_aOut + 2 * b->run[i]->nalm;
  }
  cudaEvent_t e0, e1;
  FNL_CUDA(cudaEventCreate(&e0));
  FNL_CUDA(cudaEventCreate(&e1));
  float best = 1e30f;
  int bs = cand[0][0], ba = cand[0][1];
  cudaStream_t st = b->streams[0];
  try {
    for (const auto& c : cand) {
      build_multi(b, c[0], c[1]);
      run_batch(b, z.data(), z.data(), f.data(), oT.data(), oE.data(), st);
      FNL_CUDA(cudaEventRecord(e0, st));
      for (int r = 0; r < 2; ++r) run_batch(b, z.data(), z.data(), f.data(), oT.data(), oE.data(), st);
      FNL_CUDA(cudaEventRecord(e1, st));
      FNL_CUDA(cudaEventSynchronize(e1));
      float ms = 0.f;
      FNL_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      if (ms < best) {
        best = ms;
        bs = c[0];
        ba = c[1];
      }
    }
  } catch (...) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    throw;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  build_multi(b, bs, ba);
}

}  // namespace
}  // namespace fnl

using namespace fnl;

extern "C" {

fnl_status fnl_batch_create(fnl_shells* const* shells, int n, int nstreams, fnl_batch** out) {
  fnl_batch* b = nullptr;
  fnl_status st = guard([&] {
    FNL_REQUIRE(out, "out must not be NULL");
    *out = nullptr;
    FNL_REQUIRE(shells && n >= 1 && n <= 65536, "need 1 <= n <= 65536 shells objects");
    FNL_REQUIRE(nstreams >= 0 && nstreams <= 64, "nstreams must be in [0, 64]");
    for (int i = 0; i < n; ++i) {
      check_shells(shells[i]);
      FNL_REQUIRE(shells[i]->device == shells[0]->device, "every instance must live on one device");
      FNL_REQUIRE(!shells[i]->owner, "a batch takes shells objects made by fnl_make_shells");
    }
    DeviceScope scope(shells[0]->device);
    b = new fnl_batch;
    b->device = shells[0]->device;
    b->n = n;
    b->sh.assign(shells, shells + n);
    // scratch of each instance: the object's own for its first instance, clones after
    b->run.resize(n);
    std::vector<fnl_shells*> seen;
    for (int i = 0; i < n; ++i) {
      fnl_shells* s = shells[i];
      if (std::find(seen.begin(), seen.end(), s) == seen.end() || !s->nterms) {
        seen.push_back(s);
        b->run[i] = s;
      } else {
        b->clones.push_back(clone_scratch(s));
        b->run[i] = b->clones.back();
      }
    }
    b->multi = n <= kTcMaxInst;
    for (int i = 0; i < n && b->multi; ++i)
      b->multi = b->run[i]->nterms == b->run[0]->nterms && b->run[i]->tc_split == b->run[0]->tc_split &&
                 ring_square_group(b->run[i]) > 0 && b->run[i]->nr == b->run[i]->nr_total;  // shards: streams
    FNL_CUDA(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming));
    if (b->multi) {
      b->streams.assign(1, nullptr);
      FNL_CUDA(cudaStreamCreateWithFlags(&b->streams[0], cudaStreamNonBlocking));
      b->lane.assign(n, 0);
      autotune_multi(b);
    } else {
      // instances dealt, largest first, to the least-loaded stream; instances that share
      // scratch (one object) go together
      std::vector<fnl_shells*> distinct;
      for (fnl_shells* r : b->run)
        if (std::find(distinct.begin(), distinct.end(), r) == distinct.end()) distinct.push_back(r);
      std::vector<double> load_of(distinct.size(), 0.0);
      for (int i = 0; i < n; ++i)
        load_of[std::find(distinct.begin(), distinct.end(), b->run[i]) - distinct.begin()] += work_of(b->run[i]);
      std::vector<int> idx(distinct.size());
      std::iota(idx.begin(), idx.end(), 0);
      std::stable_sort(idx.begin(), idx.end(), [&](int a, int c) { return load_of[a] > load_of[c]; });
      const int ns = std::max(1, std::min<int>(nstreams ? nstreams : 4, (int)distinct.size()));
      std::vector<double> lane_load(ns, 0.0);
      std::vector<int> lane_of(distinct.size(), 0);
      for (int k : idx) {
        const int l = (int)(std::min_element(lane_load.begin(), lane_load.end()) - lane_load.begin());
        lane_of[k] = l;
        lane_load[l] += load_of[k];
      }
      b->lane.resize(n);
      b->order.assign(ns, {});
      for (int i = 0; i < n; ++i) {
        b->lane[i] = lane_of[std::find(distinct.begin(), distinct.end(), b->run[i]) - distinct.begin()];
        b->order[b->lane[i]].push_back(i);
      }
      b->streams.assign(ns, nullptr);
      b->joins.assign(ns, nullptr);
      for (int l = 0; l < ns; ++l) {
        FNL_CUDA(cudaStreamCreateWithFlags(&b->streams[l], cudaStreamNonBlocking));
        FNL_CUDA(cudaEventCreateWithFlags(&b->joins[l], cudaEventDisableTiming));
      }
    }
    *out = b;
  });
  if (st != FNL_OK && b) free_batch(b);
  return st;
}

void fnl_batch_destroy(fnl_batch* b) {
  if (!b) return;
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(b->device);
  cudaDeviceSynchronize();
  free_batch(b);
  if (prev >= 0) cudaSetDevice(prev);
}

fnl_status fnl_batch_info(const fnl_batch* b, int* n, int* nstreams, int* lanes) {
  return guard([&] {
    FNL_REQUIRE(b, "batch is NULL");
    if (n) *n = b->n;
    if (nstreams) *nstreams = b->multi ? 0 : (int)b->streams.size();
    if (lanes)
      for (int i = 0; i < b->n; ++i) lanes[i] = b->lane[i];
  });
}

fnl_status fnl_batch_tiles(const fnl_batch* b, int* nsyn, int* nana) {
  return guard([&] {
    FNL_REQUIRE(b, "batch is NULL");
    if (nsyn) *nsyn = b->multi ? b->syn_w : 0;
    if (nana) *nana = b->multi ? b->ana_w : 0;
  });
}

fnl_status fnl_generate_batch(fnl_batch* b, const uint64_t* seeds, const uint64_t* realisations, const double* fnl,
                              double* const* aT, double* const* aE, void* stream) {
  return guard([&] {
    FNL_REQUIRE(b, "batch is NULL");
    FNL_REQUIRE(seeds && realisations && fnl && aT && aE, "seeds, realisations, fnl, aT and aE must not be NULL");
    DeviceScope scope(b->device);
    for (int i = 0; i < b->n; ++i) {
      check_dev_ptr(aT[i], "aT[i]", false);
      check_dev_ptr(aE[i], "aE[i]", false);
    }
    if (b->multi) {
      // an owner's tile shape changed since the launch arrays were built: rebuild them
      bool stale = false;
      for (int i = 0; i < b->n; ++i) stale |= owner_of(b->run[i])->tiles_version != b->versions[i];
      if (stale) build_multi(b, b->syn_w, b->ana_w);
    } else {
      for (fnl_shells* c : b->clones)
        if (c->tiles_version != c->owner->tiles_version) refresh_clone(c, c->owner);
    }
    run_batch(b, seeds, realisations, fnl, aT, aE, (cudaStream_t)stream);
  });
}

fnl_status fnl_shells_autotune(fnl_shells* sh, void* stream, int* nsyn, int* nana) {
  return guard([&] {
    check_shells(sh);
    FNL_REQUIRE(!sh->owner, "tile shapes are set on the objects fnl_make_shells made");
    DeviceScope scope(sh->device);
    cudaStream_t st = (cudaStream_t)stream;
    if (sh->nterms) {
      // candidates: 256-wide tiles (half the MMA instructions, one accumulator set) and
      // 128-wide tiles (two accumulator sets: the epilogue of one tile overlaps the MMAs of
      // the next), for each GEMM, and 96-degree analysis tiles (the quadrature epilogue's six
      // 16-degree half chunks fall two to each of a quadrant's three warps); every candidate
      // timed on whole realisations
      const int caps[2] = {256, 128}, acaps[3] = {256, 128, 96};
      cudaEvent_t e0, e1;
      FNL_CUDA(cudaEventCreate(&e0));
      FNL_CUDA(cudaEventCreate(&e1));
      float best = 1e30f;
      int bs = 256, ba = 256;
      try {
        for (int cs : caps)
          for (int ca : acaps) {
            FNL_CUDA(cudaStreamSynchronize(st));
            configure_tc(sh, cs, ca);
            run_generate(sh, 0, 0, 1.0, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, st, false);
            FNL_CUDA(cudaEventRecord(e0, st));
            for (int r = 0; r < 2; ++r)
              run_generate(sh, 0, 0, 1.0, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, st, false);
            FNL_CUDA(cudaEventRecord(e1, st));
            FNL_CUDA(cudaEventSynchronize(e1));
            float ms = 0.f;
            FNL_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            if (ms < best) {
              best = ms;
              bs = cs;
              ba = ca;
            }
          }
      } catch (...) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        throw;
      }
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      FNL_CUDA(cudaStreamSynchronize(st));
      configure_tc(sh, bs, ba);
    }
    if (nsyn) *nsyn = sh->nterms ? sh->nsyn : 64;
    if (nana) *nana = sh->nterms ? sh->nana : 64;
  });
}

fnl_status fnl_shells_gemm_work(const fnl_shells* sh, double* syn, double* ana) {
  return guard([&] {
    check_shells(sh);
    FNL_REQUIRE(sh->nterms, "the SIMT forms compute every ring pair");
    const int np = sh->npairs, ctiles = sh->Cpad / 128;
    double dense = 0.0, s = 0.0, a = 0.0;
    for (int K : sh->K) dense += (double)K * np;
    for (const TcTile& t : sh->tiles_syn_h) s += (double)t.kvalid * std::min(t.nsize, np - t.n0);
    for (const TcTile& t : sh->tiles_ana_h)
      a += (double)std::min(t.nsize, t.kvalid - t.n0) * std::max(0, np - 32 * t.kb0);
    if (syn) *syn = dense > 0 ? s / ctiles / dense : 1.0;
    if (ana) *ana = dense > 0 ? a / ctiles / dense : 1.0;
  });
}

fnl_status fnl_shells_set_tiles(fnl_shells* sh, int syn_cap, int ana_cap) {
  return guard([&] {
    check_shells(sh);
    FNL_REQUIRE(sh->nterms, "tile shapes are fixed in the FNL_FP64 and FNL_FP32 forms");
    FNL_REQUIRE(!sh->owner, "tile shapes are set on the objects fnl_make_shells made");
    DeviceScope scope(sh->device);
    FNL_CUDA(cudaDeviceSynchronize());
    configure_tc(sh, syn_cap, ana_cap);
  });
}

}  // extern "C"
