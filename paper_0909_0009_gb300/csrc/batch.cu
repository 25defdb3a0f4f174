// Batching form: many realisations of uneven l_max and N_r launched as one CUDA graph, and
// the autotuner that picks the tensor-core tile shapes of each configuration.
//
// A batch holds n instances, each a (shells object, seed, realisation, f_NL) of steps
// (i)-(v) (Sect. 2).  Instances that share a shells object share its scratch and run in
// batch order on one stream; the distinct objects are spread over up to `nstreams`
// streams, largest first (work ~ (l_max + 1)^3 N_r), so that small configurations run
// beside large ones.  Every call captures the launches of all instances (fork and join
// through events) into a graph; the first call instantiates it, later calls update the
// executable graph in place (only kernel arguments change) and launch it on the caller's
// stream, so a batch of 64 realisations costs one graph launch on the host.
#include <algorithm>
#include <numeric>
#include <vector>

#include "fnl_internal.cuh"

struct fnl_batch {
  int device = 0;
  int n = 0;
  std::vector<fnl_shells*> sh;           // per instance
  std::vector<int> lane;                 // per instance: stream index
  std::vector<std::vector<int>> order;   // per stream: instances in launch order
  std::vector<cudaStream_t> streams;     // [nstreams]; streams[0] also begins the capture
  std::vector<cudaEvent_t> joins;        // [nstreams]
  cudaEvent_t fork = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace fnl {
namespace {

void free_batch(fnl_batch* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  for (cudaEvent_t e : b->joins)
    if (e) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  for (cudaStream_t s : b->streams)
    if (s) cudaStreamDestroy(s);
  delete b;
}

double work_of(const fnl_shells* s) { return (double)(s->lmax + 1) * (s->lmax + 1) * (s->lmax + 1) * s->nr; }

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
    }
    b = new fnl_batch;
    b->device = shells[0]->device;
    b->n = n;
    b->sh.assign(shells, shells + n);
    // distinct objects, largest first, dealt to the least-loaded stream
    std::vector<fnl_shells*> distinct;
    for (fnl_shells* s : b->sh)
      if (std::find(distinct.begin(), distinct.end(), s) == distinct.end()) distinct.push_back(s);
    std::vector<double> load_of(distinct.size(), 0.0);
    for (int i = 0; i < n; ++i)
      load_of[std::find(distinct.begin(), distinct.end(), b->sh[i]) - distinct.begin()] += work_of(b->sh[i]);
    std::vector<int> idx(distinct.size());
    std::iota(idx.begin(), idx.end(), 0);
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int c) { return load_of[a] > load_of[c]; });
    const int ns = std::max(1, std::min<int>(nstreams ? nstreams : 4, (int)distinct.size()));
    std::vector<double> lane_load(ns, 0.0);
    std::vector<int> lane_of_obj(distinct.size(), 0);
    for (int k : idx) {
      const int l = (int)(std::min_element(lane_load.begin(), lane_load.end()) - lane_load.begin());
      lane_of_obj[k] = l;
      lane_load[l] += load_of[k];
    }
    b->lane.resize(n);
    b->order.assign(ns, {});
    for (int i = 0; i < n; ++i) {
      b->lane[i] = lane_of_obj[std::find(distinct.begin(), distinct.end(), b->sh[i]) - distinct.begin()];
      b->order[b->lane[i]].push_back(i);
    }
    DeviceScope scope(b->device);
    b->streams.assign(ns, nullptr);
    b->joins.assign(ns, nullptr);
    for (int l = 0; l < ns; ++l) {
      FNL_CUDA(cudaStreamCreateWithFlags(&b->streams[l], cudaStreamNonBlocking));
      FNL_CUDA(cudaEventCreateWithFlags(&b->joins[l], cudaEventDisableTiming));
    }
    FNL_CUDA(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming));
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
  for (cudaStream_t s : b->streams)
    if (s) cudaStreamSynchronize(s);
  free_batch(b);
  if (prev >= 0) cudaSetDevice(prev);
}

fnl_status fnl_batch_info(const fnl_batch* b, int* n, int* nstreams, int* lanes) {
  return guard([&] {
    FNL_REQUIRE(b, "batch is NULL");
    if (n) *n = b->n;
    if (nstreams) *nstreams = (int)b->streams.size();
    if (lanes)
      for (int i = 0; i < b->n; ++i) lanes[i] = b->lane[i];
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
    cudaStream_t cap = b->streams[0];
    cudaGraph_t graph = nullptr;
    FNL_CUDA(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
    try {
      FNL_CUDA(cudaEventRecord(b->fork, cap));
      for (size_t l = 1; l < b->streams.size(); ++l) FNL_CUDA(cudaStreamWaitEvent(b->streams[l], b->fork, 0));
      for (size_t l = 0; l < b->streams.size(); ++l) {
        for (int i : b->order[l])
          run_generate(b->sh[i], seeds[i], realisations[i], fnl[i], nullptr, aT[i], aE[i], nullptr, nullptr, nullptr,
                       nullptr, b->streams[l], false);
        if (l) {
          FNL_CUDA(cudaEventRecord(b->joins[l], b->streams[l]));
          FNL_CUDA(cudaStreamWaitEvent(cap, b->joins[l], 0));
        }
      }
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
    FNL_CUDA(cudaGraphLaunch(b->exec, (cudaStream_t)stream));
  });
}

fnl_status fnl_shells_autotune(fnl_shells* sh, void* stream, int* nsyn, int* nana) {
  return guard([&] {
    check_shells(sh);
    DeviceScope scope(sh->device);
    cudaStream_t st = (cudaStream_t)stream;
    if (sh->nterms) {
      // candidates: 256-wide tiles (half the MMA instructions, one accumulator set) and
      // 128-wide tiles (two accumulator sets: the epilogue of one tile overlaps the MMAs of
      // the next), for each GEMM; every candidate timed on whole realisations
      const int caps[2] = {256, 128};
      cudaEvent_t e0, e1;
      FNL_CUDA(cudaEventCreate(&e0));
      FNL_CUDA(cudaEventCreate(&e1));
      float best = 1e30f;
      int bs = 256, ba = 256;
      try {
        for (int cs : caps)
          for (int ca : caps) {
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

fnl_status fnl_shells_set_tiles(fnl_shells* sh, int syn_cap, int ana_cap) {
  return guard([&] {
    check_shells(sh);
    FNL_REQUIRE(sh->nterms, "tile shapes are fixed in the FNL_FP64 and FNL_FP32 forms");
    DeviceScope scope(sh->device);
    FNL_CUDA(cudaDeviceSynchronize());
    configure_tc(sh, syn_cap, ana_cap);
  });
}

}  // extern "C"
