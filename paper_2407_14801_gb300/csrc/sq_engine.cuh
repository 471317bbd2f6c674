// Host driver of the SquareSort engine: plans scratch memory, seeds the roots
// and runs rounds of kernels until every instance is sorted.  Included once
// per key type (sq_engine_<type>.cu).
#pragma once
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "sq_engine.h"
#include "sq_kernels.cuh"

namespace sq {

// ------------------------------------------------------------ statistics ---
struct StatsBox {
  std::mutex mu;
  EngineStats s{};
  std::atomic<int> profiling{0};
  // per key type (DT_U32, DT_U64, DT_F32): leaf classes sorted by the radix base case
  std::atomic<uint32_t> radix_classes[3] = {{kRadixClassesAll}, {0u}, {kRadixClassesAll}};
};
StatsBox &stats_box();

// An asynchronous run's record: where its status and graph counters land
// (page-locked), the event after them, and what its statistics need.
struct PendingRun {
  Status status;
  GraphStats gs;
};
// Takes a free record for a run on stream st (waiting for the oldest one
// when all are taken); nullptr if none can be had.  The caller enqueues the
// copies into it, then calls pending_commit.
PendingRun *pending_take(cudaStream_t st, double key_bytes, const EngineStats &per_round, uint32_t ninst,
                         char *err, size_t errlen, int *rc);
int pending_commit(PendingRun *r, cudaStream_t st, char *err, size_t errlen);

#define SQ_CU(call)                                                                   \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess) {                                                          \
      snprintf(err, errlen, "%s failed: %s", #call, cudaGetErrorString(e_));         \
      return 5; /* SQ_ERR_CUDA */                                                     \
    }                                                                                 \
  } while (0)

template <int DT>
struct Engine {
  typedef KT<DT> K;
  typedef typename K::elem_t E;
  static constexpr int NCLASS = LeafCfg<DT>::nclass;
  static constexpr int SKEW_CAP = sizeof(E) == 8 ? 2048 : 1024;
  static constexpr size_t KEY_BYTES = sizeof(typename K::key_t);
  // Leaf sorts of float32 keys use the one-word element (NaN bits restored
  // by the leaf kernels, or the leaf left to the fix list).
  static constexpr int LDT = DT == DT_F32 ? DT_F32W : DT;
  typedef KT<LDT> KL;
  typedef typename KL::elem_t EL;
  static constexpr bool kFix = KL::lossy;  // NaN-heavy float32 leaves go to the fix list
  static constexpr u32 kHostExpandCols = 2048;  // roots with this many columns are expanded on the host

  static u32 max_leaf() { return class_cap(NCLASS - 1); }
  static u32 max_pivots() { return LeafCfg<DT>::max_pivots; }  // one CTA's pivot sample
  // the largest pivot sample of any node (a cluster's, where the key type has one)
  static u32 max_sample() { return std::max(LeafCfg<DT>::max_pivots, LeafCfg<DT>::max_pivots_big); }
  // the largest n: (max_sample() + 1)^2, within 32-bit node sizes
  static u64 max_n() { return std::min<u64>((u64)(max_sample() + 1) * (max_sample() + 1), 0xffffffffull); }

  // ---- launch helpers ---------------------------------------------------
  struct Launcher {
    cudaStream_t st;
    bool prof;
    EngineStats local{};
    std::vector<cudaEvent_t> evs;
    std::vector<int> fam;
    void begin(int f) {
      local.launches[f]++;
      if (prof) {
        cudaEvent_t a;
        cudaEventCreate(&a);
        cudaEventRecord(a, st);
        evs.push_back(a);
        fam.push_back(f);
      }
    }
    void end() {
      if (prof) {
        cudaEvent_t b;
        cudaEventCreate(&b);
        cudaEventRecord(b, st);
        evs.push_back(b);
      }
    }
    void collect() {  // after a stream synchronize
      for (size_t i = 0; i + 1 < evs.size(); i += 2) {
        float ms = 0;
        cudaEventElapsedTime(&ms, evs[i], evs[i + 1]);
        local.ms[fam[i / 2]] += ms;
        cudaEventDestroy(evs[i]);
        cudaEventDestroy(evs[i + 1]);
      }
      evs.clear();
      fam.clear();
    }
  };

  // The 48 KiB default covers static plus dynamic shared memory, so any
  // sizeable dynamic request raises the kernel's limit first.
  template <class Kern>
  static cudaError_t set_smem(Kern kern, size_t bytes) {
    if (bytes <= 32 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  }

  // Grid of a launch whose item count the kernel reads on the device: enough
  // CTAs (or clusters) to fill every SM; the kernel strides over its list.
  template <class Kern>
  static u32 fill_grid(Kern kern, int threads, size_t smem, int nsm) {
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, smem) != cudaSuccess || occ < 1) occ = 1;
    return (u32)occ * (u32)nsm;
  }
  template <class Kern>
  static u32 fill_clusters(Kern kern, int threads, size_t smem, int G, int nsm) {
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3((unsigned)(G * std::max(1, nsm / G)), 1, 1);
    cfg.blockDim = dim3(threads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = G;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int ncl = 0;
    if (cudaOccupancyMaxActiveClusters(&ncl, kern, &cfg) != cudaSuccess || ncl < 1) ncl = std::max(1, nsm / G);
    return (u32)ncl * (u32)G;
  }

  template <int T, int R, bool WARP>
  static cudaError_t launch_leaf(Launcher &L, const Ctx *cp, int cls, u32 count, int nsm) {
    const size_t smem = leaf_sort_bytes<LDT, T, R, WARP>() + (KL::lossy ? (WARP ? 8 : 1) * 4 * kNanWords : 0);
    auto kern = k_leaf<LDT, T, R, WARP>;
    cudaError_t e = set_smem(kern, smem);
    if (e != cudaSuccess) return e;
    const int threads = WARP ? 256 : T;
    const u32 grid = count == kDev ? fill_grid(kern, threads, smem, nsm) : (WARP ? (count + 7) / 8 : count);
    L.begin(KF_LEAF);
    kern<<<grid, threads, smem, L.st>>>(cp, cls, count);
    L.end();
    return cudaGetLastError();
  }

  template <class Kern, class... Args>
  static cudaError_t launch_cluster(Kern kern, dim3 grid, int T, size_t smem, int G, cudaStream_t st,
                                    Args... args) {
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = grid;
    cfg.blockDim = dim3(T, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = G;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, kern, args...);
    return e != cudaSuccess ? e : cudaGetLastError();
  }

  template <int T, int R, int G>
  static cudaError_t launch_leaf_cluster(Launcher &L, const Ctx *cp, int cls, u32 count, int nsm) {
    const size_t smem = leaf_sort_bytes<LDT, T, R, false>() + (KL::lossy ? 4 * kNanWords : 0);
    auto kern = k_leaf_cluster<LDT, T, R, G>;
    cudaError_t e = set_smem(kern, smem);
    if (e != cudaSuccess) return e;
    const u32 grid = count == kDev ? fill_clusters(kern, T, smem, G, nsm) : count * G;
    L.begin(KF_LEAF);
    e = launch_cluster(kern, dim3(grid, 1, 1), T, smem, G, L.st, cp, cls, count);
    L.end();
    return e;
  }

  // Leaves of 32-bit key ordinals (uint32, float32) take the radix base case
  // in the classes where it is faster than the merge sort.
  static constexpr bool kRadix = sizeof(EL) == 8 && KL::top_is_value;

  template <int T, int R>
  static cudaError_t launch_leaf_radix(Launcher &L, const Ctx *cp, int cls, u32 count, int nsm) {
    const size_t smem = radix_leaf_bytes<LDT, T, R>();
    auto kern = k_leaf_radix<LDT, T, R>;
    cudaError_t e = set_smem(kern, smem);
    if (e != cudaSuccess) return e;
    const u32 grid = count == kDev ? fill_grid(kern, T, smem, nsm) : count;
    L.begin(KF_LEAF);
    kern<<<grid, T, smem, L.st>>>(cp, cls, count);
    L.end();
    return cudaGetLastError();
  }

  template <int T, int R, int G>
  static cudaError_t launch_leaf_radix_cluster(Launcher &L, const Ctx *cp, int cls, u32 count, int nsm) {
    const size_t smem = radix_leaf_bytes<LDT, T, R>();
    auto kern = k_leaf_radix_cluster<LDT, T, R, G>;
    cudaError_t e = set_smem(kern, smem);
    if (e != cudaSuccess) return e;
    const u32 grid = count == kDev ? fill_clusters(kern, T, smem, G, nsm) : count * G;
    L.begin(KF_LEAF);
    e = launch_cluster(kern, dim3(grid, 1, 1), T, smem, G, L.st, cp, cls, count);
    L.end();
    return e;
  }

  static u32 radix_classes() { return kRadix ? stats_box().radix_classes[DT].load() & kRadixClassesAll : 0u; }

  static cudaError_t launch_leaf_class(Launcher &L, const Ctx *cp, int cls, u32 count, int nsm) {
    if constexpr (kRadix) {
      if ((radix_classes() >> cls) & 1u) switch (cls) {  // (class c holds 2K, 8K, then (c - 2) * 8192 elements)
        case 2: return launch_leaf_radix<128, 16>(L, cp, 2, count, nsm);
        case 3: return launch_leaf_radix<512, 16>(L, cp, 3, count, nsm);
        case 4: return launch_leaf_radix<512, 32>(L, cp, 4, count, nsm);
        case 5:
        case 6: return launch_leaf_radix_cluster<512, 32, 2>(L, cp, cls, count, nsm);
        case 7:
        case 8: return launch_leaf_radix_cluster<512, 32, 3>(L, cp, cls, count, nsm);
        case 9:
        case 10: return launch_leaf_radix_cluster<512, 32, 4>(L, cp, cls, count, nsm);
        default: break;
      }
    }
    switch (cls) {
      case 0: return launch_leaf<32, 2, true>(L, cp, 0, count, nsm);
      case 1: return launch_leaf<32, 16, true>(L, cp, 1, count, nsm);
      case 2: return launch_leaf<128, 16, false>(L, cp, 2, count, nsm);
      case 3: return launch_leaf<512, 16, false>(L, cp, 3, count, nsm);
      case 4: return launch_leaf_cluster<512, 16, 2>(L, cp, 4, count, nsm);
      case 5: return launch_leaf_cluster<512, 16, 3>(L, cp, 5, count, nsm);
      case 6: return launch_leaf_cluster<512, 16, 4>(L, cp, 6, count, nsm);
      case 7: return launch_leaf_cluster<512, 16, 5>(L, cp, 7, count, nsm);
      case 8: return launch_leaf_cluster<512, 16, 6>(L, cp, 8, count, nsm);
      case 9: return launch_leaf_cluster<512, 16, 7>(L, cp, 9, count, nsm);
      default: return launch_leaf_cluster<512, 16, 8>(L, cp, 10, count, nsm);
    }
  }

  // The (key, val) merge sort of this round's fix list.
  static cudaError_t launch_fixup(Launcher &L, const Ctx *cp, int nsm) {
    constexpr bool wide = sizeof(E) == 8;
    constexpr int T = wide ? 1024 : 512, R = 16, G = wide ? 4 : 8;
    const size_t smem = sizeof(E) * (size_t)Sorter<K, T, R, false>::SMEM;
    auto kern = k_fixup<DT, T, R, G>;
    cudaError_t e = set_smem(kern, smem);
    if (e != cudaSuccess) return e;
    L.begin(KF_AUX);
    e = launch_cluster(kern, dim3(std::max(1, nsm / G) * G, 1, 1), T, smem, G, L.st, cp);
    L.end();
    return e;
  }

  template <int T, int R, bool WARP>
  static cudaError_t launch_pivots(Launcher &L, const Ctx *cp, u32 ready, u32 pmin, u32 pmax, int nsm) {
    typedef Sorter<K, T, R, WARP> S;
    const size_t smem = (size_t)(WARP ? 8 : 1) * S::SMEM * sizeof(E);
    auto kern = k_pivots<DT, T, R, WARP>;
    cudaError_t e = set_smem(kern, smem);
    if (e != cudaSuccess) return e;
    const int threads = WARP ? 256 : T;
    const u32 grid = ready == kDev ? fill_grid(kern, threads, smem, nsm) : (WARP ? (ready + 7) / 8 : ready);
    L.begin(KF_PIVOTS);
    kern<<<grid, threads, smem, L.st>>>(cp, ready, pmin, pmax);
    L.end();
    return cudaGetLastError();
  }

  static cudaError_t launch_all_pivots(Launcher &L, const Ctx *cp, u32 ready, u32 max_k, int nsm) {
    cudaError_t e = cudaSuccess;
    const u32 maxp = max_k;  // (an appendix-variant node sorts k samples, one more than its pivots)
    e = launch_pivots<32, 16, true>(L, cp, ready, 0, 512, nsm);
    if (e == cudaSuccess && maxp > 512) e = launch_pivots<128, 16, false>(L, cp, ready, 512, 2048, nsm);
    if (e == cudaSuccess && maxp > 2048) e = launch_pivots<512, 16, false>(L, cp, ready, 2048, 8192, nsm);
    if constexpr (LeafCfg<DT>::max_pivots > 8192)
      if (e == cudaSuccess && maxp > 8192) e = launch_pivots<1024, 16, false>(L, cp, ready, 8192, 16384, nsm);
    if constexpr (LeafCfg<DT>::max_pivots_big > 0)
      if (e == cudaSuccess && maxp > LeafCfg<DT>::max_pivots + 1) e = launch_pivots_cluster(L, cp, ready, nsm);
    return e;
  }

  // Samples larger than one CTA sorts: a cluster of 8 CTAs per node.
  static cudaError_t launch_pivots_cluster(Launcher &L, const Ctx *cp, u32 ready, int nsm) {
    constexpr int G = 8;
    const size_t smem = (size_t)Sorter<K, 512, 16, false>::SMEM * sizeof(E);
    auto kern = k_pivots_cluster<DT>;
    cudaError_t e = set_smem(kern, smem);
    if (e != cudaSuccess) return e;
    const u32 ncl = std::max<u32>(1, ready == kDev ? (u32)(nsm / G) : std::min<u32>(ready, (u32)(nsm / G)));
    L.begin(KF_PIVOTS);
    e = launch_cluster(kern, dim3(G * ncl, 1, 1), 512, smem, G, L.st, cp, ready, (u32)LeafCfg<DT>::max_pivots);
    L.end();
    return e;
  }

  // ---- one round ----------------------------------------------------------
  // Leaves (simple_sort), then for the ready nodes the plan, pivots, counts,
  // bucket starts, SkewTranspose and bucket children, then the column
  // children of new nodes.  hc: the round's counts when the host drives the
  // rounds (launches sized to them, empty steps skipped); null for a graph
  // round, whose kernels read the counts on the device.
  struct RoundArgs {
    int nsm;
    int skew_only;
    const void *piv_keys;
    const u32 *piv_vals;
    u64 *bucket_start;
    u64 k;
    double skew_elems;  // skew_only: elements moved
    int tags;           // every instance has tag scratch
    u32 kmax;           // graph rounds: the largest k of any node of the run
  };

  static cudaError_t issue_round(Launcher &L, const Ctx *cp, const Counters *hc, const RoundArgs &A) {
    const cudaStream_t st = L.st;
    const int nsm = A.nsm;
    const int grid_count = nsm * 2, grid_scan = nsm * 8, grid_skew = nsm * 5, grid_skew_tags = nsm * (32 / SQ_SKEW_WARPS),
              grid_expand = nsm * 4;
    cudaError_t e;
#define SQ_TRY(x)                      \
  do {                                 \
    if ((e = (x)) != cudaSuccess) return e; \
  } while (0)
    L.begin(KF_AUX);
    k_round_begin<<<1, 64, 0, st>>>(cp);
    L.end();
    SQ_TRY(cudaGetLastError());
    bool any_leaves = false;
    for (int cl = 0; cl < NCLASS; cl++) {
      const u32 n = hc ? hc->leaves[cl] : kDev;
      if (!n) continue;
      if (hc) L.local.bytes[KF_LEAF] += 2.0 * (KEY_BYTES + 4) * (double)hc->leaf_elems[cl];
      SQ_TRY(launch_leaf_class(L, cp, cl, n, nsm));
      any_leaves = true;
    }
    if (kFix && any_leaves) SQ_TRY(launch_fixup(L, cp, nsm));
    const u32 ready = hc ? hc->ready : kDev;
    if (ready) {
      const double re = A.skew_only ? A.skew_elems : (hc ? (double)hc->ready_elems : 0.0);
      if (hc) L.local.nodes += A.skew_only ? 0 : ready;
      L.begin(KF_PLAN);
      k_plan<<<1, 1024, 0, st>>>(cp, ready, K::key_words);
      L.end();
      SQ_TRY(cudaGetLastError());
      const u32 kmax = hc ? std::max<u32>(hc->max_ready_k, 2) : A.kmax;
      if (A.skew_only) {
        L.begin(KF_AUX);
        k_put_pivots<DT><<<((u32)A.k + 255) / 256, 256, 0, st>>>(cp, (const typename K::key_t *)A.piv_keys,
                                                                  A.piv_vals);
        L.end();
        SQ_TRY(cudaGetLastError());
      } else {
        SQ_TRY(launch_all_pivots(L, cp, ready, kmax, nsm));
      }
      // nodes with up to kCountSmemPivots pivots: pivots and totals in shared
      // memory; larger ones (a launch of their own): in global memory
      const u32 kms = std::min<u32>(kmax, kCountSmemPivots + 1);
      const size_t smem_count = (size_t)(kms - 1) * sizeof(E) + (size_t)kms * 4;
      SQ_TRY(set_smem(k_count<DT, false>, smem_count));
      L.begin(KF_COUNT);
      k_count<DT, false><<<grid_count, 1024, smem_count, st>>>(cp, ready, kms);
      if (kmax - 1 > kCountSmemPivots) k_count<DT, true><<<grid_count, 1024, 0, st>>>(cp, ready, 1u);
      L.end();
      L.local.bytes[KF_COUNT] += (KEY_BYTES + 4) * re;
      SQ_TRY(cudaGetLastError());
      L.begin(KF_SCAN);
      k_scan<<<grid_scan, 256, 0, st>>>(cp, ready, K::key_words);
      L.end();
      SQ_TRY(cudaGetLastError());
      L.begin(KF_BSTART);
      k_bstart<<<hc ? ready : (u32)nsm * 2, 1024, 0, st>>>(cp, ready, K::key_words);
      L.end();
      SQ_TRY(cudaGetLastError());
      const size_t smem_skew = sizeof(SkewSmem<DT, SKEW_CAP>);
      L.begin(KF_SKEW);
      if (A.tags) {  // every instance has tag scratch: a counting sort by the count's tags
        constexpr int CAP_T = 256 * SQ_SKEW_WARPS;  // 256 elements a warp per chunk
        const size_t smem_tags = sizeof(SkewTagSmem<DT, CAP_T>);
        SQ_TRY(set_smem(k_skew_tags<DT, CAP_T>, smem_tags));
        k_skew_tags<DT, CAP_T><<<grid_skew_tags, 32 * SQ_SKEW_WARPS, smem_tags, st>>>(cp, ready);
        SQ_TRY(cudaGetLastError());
        L.end();
        L.begin(KF_SKEW);
        k_copy_runs<DT><<<nsm * 4, 256, 0, st>>>(cp);  // (returns at once when no run was queued)
      } else {
        SQ_TRY(set_smem(k_skew<DT, SKEW_CAP, false>, smem_skew));
        k_skew<DT, SKEW_CAP, false><<<grid_skew, 256, smem_skew, st>>>(cp, ready);
      }
      L.end();
      L.local.bytes[KF_SKEW] += 2.0 * (KEY_BYTES + 4) * re;
      SQ_TRY(cudaGetLastError());
      if (A.skew_only) {
        L.begin(KF_AUX);
        k_get_bstart<DT><<<((u32)A.k + 256) / 256, 256, 0, st>>>(cp, A.bucket_start);
        L.end();
        SQ_TRY(cudaGetLastError());
      } else {
        L.begin(KF_EXPAND);
        k_expand_buckets<DT><<<grid_expand, 256, 0, st>>>(cp, ready);
        L.end();
        SQ_TRY(cudaGetLastError());
      }
    }
    if (!A.skew_only && (!hc || ready || hc->fresh)) {
      L.begin(KF_EXPAND);
      k_expand_cols<DT><<<grid_expand, 256, 0, st>>>(cp);
      L.end();
      SQ_TRY(cudaGetLastError());
    }
#undef SQ_TRY
    return cudaSuccess;
  }

  // Pinned host memory (512 bytes) for the round read-backs, one buffer per
  // thread, allocated on first use and kept: pinning per call costs more
  // than a whole small sort.
  static cudaError_t pinned_readback(void **out) {
    struct Pinned {
      void *p = nullptr;
      ~Pinned() {
        if (p) cudaFreeHost(p);
      }
    };
    static thread_local Pinned buf;
    if (!buf.p) {
      const cudaError_t e = cudaMallocHost(&buf.p, 512);
      if (e != cudaSuccess) {
        buf.p = nullptr;
        return e;
      }
    }
    *out = buf.p;
    return cudaSuccess;
  }

  // ---- CUDA-graph rounds ----------------------------------------------------
  // The recursion as one graph launch: a device-side while loop whose body is
  // two rounds (the even and the odd parity of the double-buffered lists), the
  // second under a condition, each ended by k_round_end, which sets the
  // conditions.  Every launch reads its context from ctx[0] (the first round
  // of the body) or ctx[1] and its item counts from the device, so one
  // instantiated graph serves every run of this key type on this thread.
  struct GraphSlot {
    int dev = -1, nsm = 0;
    u32 radix = 0;  // the radix classes the captured leaf launches follow
    cudaStream_t last = nullptr;  // stream of the last launch (its context buffer is this slot's)
    Ctx *ctx = nullptr;  // device, 2 contexts
    GraphStats *gs = nullptr;
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    EngineStats per_round{};  // launches of one round, by family
    void reset() {
      if (exec) cudaGraphExecDestroy(exec);
      if (graph) cudaGraphDestroy(graph);
      if (cap) cudaStreamDestroy(cap);
      if (ctx) cudaFree(ctx);
      exec = nullptr;
      graph = nullptr;
      cap = nullptr;
      ctx = nullptr;
      gs = nullptr;
      dev = -1;
    }
    ~GraphSlot() { reset(); }
  };
  // One graph per bound on the nodes' k (a power of two, so that the count
  // kernel's shared memory and the pivot-sort launches fit the run).
  static GraphSlot &graph_slot(int kb) {  // kb <= 16: k <= max_sample() + 1 <= 2^16
    static thread_local GraphSlot s[17];
    return s[kb];
  }

  static constexpr unsigned long long kMaxRounds = 4096;  // far above any recursion depth

  // Builds (once per thread, device and instance count) the graph of rounds.
  static int graph_prepare(GraphSlot &G, int dev, int nsm, u32 kmax, char *err, size_t errlen) {
    if (G.exec && G.dev == dev && G.radix == radix_classes()) return 0;
    G.reset();
    G.radix = radix_classes();
    SQ_CU(cudaMalloc((void **)&G.ctx, 2 * sizeof(Ctx) + sizeof(GraphStats)));
    G.gs = reinterpret_cast<GraphStats *>(G.ctx + 2);
    SQ_CU(cudaStreamCreateWithFlags(&G.cap, cudaStreamNonBlocking));
    SQ_CU(cudaGraphCreate(&G.graph, 0));
    cudaGraphConditionalHandle loop, second;
    SQ_CU(cudaGraphConditionalHandleCreate(&loop, G.graph, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams wp = {};
    wp.type = cudaGraphNodeTypeConditional;
    wp.conditional.handle = loop;
    wp.conditional.type = cudaGraphCondTypeWhile;
    wp.conditional.size = 1;
    cudaGraphNode_t wnode;
    SQ_CU(cudaGraphAddNode(&wnode, G.graph, nullptr, nullptr, 0, &wp));
    cudaGraph_t body = wp.conditional.phGraph_out[0];
    SQ_CU(cudaGraphConditionalHandleCreate(&second, body, 0, 0));
    Launcher L;
    L.st = G.cap;
    L.prof = false;
    RoundArgs A;
    memset(&A, 0, sizeof(A));
    A.nsm = nsm;
    A.tags = 1;  // graph runs are sorts whose instances all carry tag scratch
    A.kmax = kmax;
    // first round of the body, then the conditional second round
    SQ_CU(cudaStreamBeginCaptureToGraph(G.cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    cudaError_t ce = issue_round(L, G.ctx, nullptr, A);
    if (ce == cudaSuccess) {
      k_round_end<<<1, 1, 0, G.cap>>>(G.ctx, loop, second, 1, G.gs, kMaxRounds);
      ce = cudaGetLastError();
    }
    // the captured round's last node(s): the conditional second round follows them
    std::vector<cudaGraphNode_t> tail;
    if (ce == cudaSuccess) {
      cudaStreamCaptureStatus cs;
      const cudaGraphNode_t *deps = nullptr;
      size_t nl = 0;
      ce = cudaStreamGetCaptureInfo(G.cap, &cs, nullptr, nullptr, &deps, nullptr, &nl);
      if (ce == cudaSuccess) tail.assign(deps, deps + nl);
    }
    cudaGraph_t got = nullptr;
    cudaError_t ee = cudaStreamEndCapture(G.cap, &got);
    SQ_CU(ce);
    SQ_CU(ee);
    const size_t nl = tail.size();
    cudaGraphNodeParams ip = {};
    ip.type = cudaGraphNodeTypeConditional;
    ip.conditional.handle = second;
    ip.conditional.type = cudaGraphCondTypeIf;
    ip.conditional.size = 1;
    cudaGraphNode_t inode;
    SQ_CU(cudaGraphAddNode(&inode, body, tail.data(), nullptr, nl, &ip));
    cudaGraph_t body2 = ip.conditional.phGraph_out[0];
    SQ_CU(cudaStreamBeginCaptureToGraph(G.cap, body2, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    ce = issue_round(L, G.ctx + 1, nullptr, A);
    if (ce == cudaSuccess) {
      k_round_end<<<1, 1, 0, G.cap>>>(G.ctx + 1, loop, second, 0, G.gs, kMaxRounds);
      ce = cudaGetLastError();
    }
    ee = cudaStreamEndCapture(G.cap, &got);
    SQ_CU(ce);
    SQ_CU(ee);
    SQ_CU(cudaGraphInstantiate(&G.exec, G.graph, 0));
    for (int f = 0; f < KF_COUNT_FAMILIES; f++) G.per_round.launches[f] = L.local.launches[f] / 2;
    G.dev = dev;
    G.nsm = nsm;
    return 0;
  }

  // ---- scratch plan: list capacities (proven bounds) and slab layout ------
  struct Plan {
    u32 leaf_cap[kLeafClasses];
    u64 ready_cap, fresh_cap, node_cap, meta_cap;
    size_t o_inst, o_leaves[2][kLeafClasses], o_ready[2], o_fresh[2], o_cnt, o_status, o_meta, o_done, o_trace,
        o_wbase, o_fix, o_runs, o_ctx;
    u64 fix_cap, runs_cap;
    size_t slab_bytes;
  };

  // Leaves made in one round cover disjoint ranges and come from the columns
  // or buckets of nodes with n > cutoff (at most 2*ceil(sqrt n) each), so a
  // round makes at most 2*(N/floor(sqrt c) + N/c) of them; ready nodes
  // (n > c, disjoint) number at most N/(c+1), new nodes twice that.
  // cutoff: the smallest cutoff of the run's instances (bounds the counts of
  // leaves and nodes); cutoff_max: the largest (bounds the leaf classes).
  static Plan make_plan(u64 total_n, u32 ninst, u32 cutoff, u32 cutoff_max, u32 trace_cap, int skew_only, u32 k,
                        u32 cols) {
    Plan P;
    const double sc = std::floor(std::sqrt((double)cutoff));
    const u64 leaf_bound = (u64)(2.0 * ((double)total_n / sc + (double)total_n / cutoff)) + 2ull * ninst + 64;
    for (int c = 0; c < kLeafClasses; c++) {
      const u64 lo = c == 0 ? 1 : (u64)class_cap(c - 1) + 1;
      u64 cap = std::min<u64>(leaf_bound, total_n / lo + ninst + 64);
      if (lo > cutoff_max || c >= NCLASS) cap = 0;  // no leaf of this class can exist
      P.leaf_cap[c] = (u32)std::min<u64>(cap, 0xffffffffull);
    }
    P.ready_cap = total_n / (cutoff + 1) + ninst + 64;
    P.fresh_cap = 2 * (total_n / (cutoff + 1)) + ninst + 64;
    P.node_cap = std::max<u64>(1024, 2 * P.fresh_cap + ninst);
    const double kw = (double)K::key_words;
    P.meta_cap = (u64)((double)total_n * (1.0 / kCountCols + 1.0 / kSkewBkts) +
                       (6.0 + kw) * ((double)total_n / std::sqrt((double)cutoff + 1) + P.ready_cap)) +
                 32 * P.ready_cap + 4096;
    if (skew_only) {  // one node, no leaves, no children
      for (int c = 0; c < kLeafClasses; c++) P.leaf_cap[c] = 0;
      P.node_cap = 1;
      P.ready_cap = P.fresh_cap = 1;
      P.meta_cap = meta_layout(k, cols, (cols + kCountCols - 1) / kCountCols, (k + kSkewBkts - 1) / kSkewBkts,
                               K::key_words)
                       .total +
                   64;
    }
    size_t off = 0;
    auto carve = [&](size_t bytes) {
      const size_t o = off;
      off += (bytes + 255) & ~(size_t)255;
      return o;
    };
    P.o_inst = carve(sizeof(Inst) * std::max<u32>(ninst, 1));
    for (int q = 0; q < 2; q++)
      for (int c = 0; c < kLeafClasses; c++) P.o_leaves[q][c] = carve(sizeof(Leaf) * (size_t)P.leaf_cap[c]);
    P.o_ready[0] = carve(4 * P.ready_cap);
    P.o_ready[1] = carve(4 * P.ready_cap);
    P.o_fresh[0] = carve(4 * P.fresh_cap);
    P.o_fresh[1] = carve(4 * P.fresh_cap);
    P.o_cnt = carve(2 * sizeof(Counters));
    P.o_status = carve(sizeof(Status));
    P.o_meta = carve(4 * P.meta_cap);
    P.o_done = carve(4 * (size_t)std::max<u32>(ninst, 1));
    P.o_trace = carve(sizeof(TraceRec) * (size_t)trace_cap);
    P.o_wbase = carve(4 * 4 * P.ready_cap);
    P.fix_cap = 0;  // any leaf of a lossy element type may go to the fix list
    if (kFix)
      for (int c = 0; c < kLeafClasses; c++) P.fix_cap += P.leaf_cap[c];
    P.o_fix = carve(sizeof(Leaf) * (size_t)P.fix_cap);
    // run copies of big SkewTranspose tiles (a full list only makes the
    // SkewTranspose copy its runs itself)
    P.runs_cap = skew_only ? 0 : std::min<u64>(total_n / 256 + 4096, 0xffffffffull);
    P.o_runs = carve(sizeof(RunCopy) * (size_t)P.runs_cap);
    P.o_ctx = carve(2 * sizeof(Ctx));
    P.slab_bytes = off;
    return P;
  }

  static u64 skew_scratch_bytes(u64 n, u32 cols, u32 k) {
    const Plan P = make_plan(n, 1, 2, 2, 0, 1, k, cols);
    return ((P.slab_bytes + 255) & ~(u64)255) + ((sizeof(Node) + 255) & ~(u64)255);
  }

  static u64 scratch_bytes(u64 total_n, u32 ninst, u32 cutoff, u32 cutoff_max) {
    const Plan P = make_plan(total_n, ninst, cutoff, std::max(cutoff, cutoff_max), 0, 0, 0, 0);
    return P.slab_bytes + sizeof(Node) * P.node_cap + 4096;
  }

  // ---- one run ------------------------------------------------------------
  static int run(const RunSpec &spec, cudaStream_t st, char *err, size_t errlen) {
    const u32 ninst = spec.ninst;
    auto cutoff_of = [&](u32 i) { return spec.inst[i].cutoff ? spec.inst[i].cutoff : spec.cutoff; };
    u32 cutoff = ninst ? 0xffffffffu : spec.cutoff;  // the smallest cutoff bounds the work lists
    u32 cutoff_max = spec.cutoff;
    for (u32 i = 0; i < ninst; i++) {
      const u32 ci = cutoff_of(i);
      if (ci < 2 || ci > max_leaf()) {
        snprintf(err, errlen, "cutoff %u outside [2, %u]", ci, max_leaf());
        return 1;
      }
      cutoff = std::min(cutoff, ci);
      cutoff_max = std::max(cutoff_max, ci);
    }
    if (cutoff < 2) {
      snprintf(err, errlen, "cutoff %u outside [2, %u]", cutoff, max_leaf());
      return 1;
    }
    int dev = 0, nsm = 0;
    SQ_CU(cudaGetDevice(&dev));
    SQ_CU(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));

    // ---- sizes
    u64 total_n = 0, max_n = 0;
    for (u32 i = 0; i < ninst; i++) {
      total_n += spec.inst[i].n;
      max_n = std::max<u64>(max_n, spec.inst[i].n);
    }
    const u64 lim = Engine::max_n();
    if (!spec.skew_only && max_n > lim) {
      snprintf(err, errlen, "n = %llu exceeds the largest supported size %llu for this key type",
               (unsigned long long)max_n, (unsigned long long)lim);
      return 1;
    }
    const u64 vlim = (u64)(max_pivots() + 1) * (max_pivots() + 1);  // the variant sorts its k samples in one CTA
    for (u32 i = 0; i < ninst && !spec.skew_only; i++)
      if (spec.inst[i].variant &&
          (spec.inst[i].n >= vlim || cutoff_of(i) < 8 || (DT != DT_U32 && DT != DT_U64))) {
        snprintf(err, errlen, "the appendix variant takes integer keys, n < %llu and a cutoff >= 8",
                 (unsigned long long)vlim);
        return 1;
      }
    const Plan P = make_plan(total_n, ninst, cutoff, cutoff_max, spec.trace_cap, spec.skew_only, (u32)spec.k, (u32)spec.cols);
    u32 leaf_cap[kLeafClasses];
    for (int cl = 0; cl < kLeafClasses; cl++) leaf_cap[cl] = P.leaf_cap[cl];
    const u64 ready_cap = P.ready_cap, fresh_cap = P.fresh_cap, meta_cap = P.meta_cap;
    u64 node_cap = P.node_cap;
    // An asynchronous run cannot stop for the host to grow the node pool, so
    // it starts with room for 4 * total_n / cutoff + 4096 recursing nodes
    // (measured peak, over sizes 2^10..2^28 and cutoffs 64..65536: under
    // 2 * n / cutoff), and runs synchronously when that pool would be large.
    bool async = spec.async && spec.graph && !spec.skew_only && !spec.trace_cap &&
                 stats_box().profiling.load() == 0;
    if (async) {
      const u64 want = 4 * (total_n / cutoff) + 4096 + 2 * fresh_cap + ninst;
      if (want * sizeof(Node) > (1ull << 30) || want > 0xffffffffull)
        async = false;
      else
        node_cap = std::max(node_cap, want);
    }
    const size_t off = P.slab_bytes, o_inst = P.o_inst, o_ready[2] = {P.o_ready[0], P.o_ready[1]};
    const size_t o_fresh[2] = {P.o_fresh[0], P.o_fresh[1]}, o_cnt = P.o_cnt, o_status = P.o_status;
    const size_t o_meta = P.o_meta, o_done = P.o_done, o_trace = P.o_trace, o_wbase = P.o_wbase;
    size_t o_leaves[2][kLeafClasses];
    for (int q = 0; q < 2; q++)
      for (int cl = 0; cl < kLeafClasses; cl++) o_leaves[q][cl] = P.o_leaves[q][cl];
    char *slab = nullptr;
    Node *nodes = nullptr;
    u32 *samp = nullptr;
    auto dalloc = [&](void **p, size_t bytes) -> cudaError_t {
      if (spec.dev_alloc) {
        *p = spec.dev_alloc(spec.alloc_ctx, bytes);
        return *p ? cudaSuccess : cudaErrorMemoryAllocation;
      }
      return cudaMallocAsync(p, bytes, st);
    };
    struct Free {
      const RunSpec &spec;
      cudaStream_t st;
      char **slab;
      Node **nodes;
      u32 **samp;
      void rel(void *p) {
        if (!p) return;
        if (spec.dev_free)
          spec.dev_free(spec.alloc_ctx, p);
        else
          cudaFreeAsync(p, st);
      }
      ~Free() {
        rel(*slab);
        rel(*nodes);
        rel(*samp);
      }
    } free_guard{spec, st, &slab, &nodes, &samp};
    SQ_CU(dalloc((void **)&slab, off));
    SQ_CU(dalloc((void **)&nodes, sizeof(Node) * node_cap));
    // Appendix variant: the store for the pivot samples of nodes whose
    // columns recurse (drawn at expansion, read at the pivot step).  Such a
    // node keeps floor(sqrt n) samples, at most 3n/cutoff (its m or its last
    // column, at most 3m+1 elements, exceeds the cutoff), and the nodes of one
    // depth are disjoint; min(8, 24/cutoff) * n covers the totals measured
    // over cutoffs 3..64 (3.9 n at cutoff 3) with room to spare.  A run that
    // needs more stops with the sample-store error.
    u64 samp_cap = 0;
    {
      u64 var_n = 0;
      u32 var_cut = 0xffffffffu;
      for (u32 i = 0; i < ninst; i++)
        if (spec.inst[i].variant) {
          var_n += spec.inst[i].n;
          var_cut = std::min(var_cut, cutoff_of(i));
        }
      if (var_n) {
        const double per = std::min(8.0, 24.0 / (double)var_cut);
        const u64 elems = (u64)(per * (double)var_n) + 4 * (u64)std::sqrt((double)var_n) + 4096;
        samp_cap = elems * (K::key_words + 1) + 2;
        SQ_CU(dalloc((void **)&samp, 4 * samp_cap));
      }
    }

    Ctx c;
    memset(&c, 0, sizeof(c));
    c.inst = (Inst *)(slab + o_inst);
    c.nodes = nodes;
    c.node_cap = (u32)node_cap;
    for (int cl = 0; cl < kLeafClasses; cl++) c.leaf_cap[cl] = leaf_cap[cl];
    c.ready_cap = (u32)ready_cap;
    c.wbase = (u32 *)(slab + o_wbase);
    c.fix = (Leaf *)(slab + P.o_fix);
    c.fix_cap = (u32)std::min<u64>(P.fix_cap, 0xffffffffull);
    c.runs = (RunCopy *)(slab + P.o_runs);
    c.runs_cap = (u32)P.runs_cap;
    c.samp = samp;
    c.samp_cap = samp_cap;
    c.fresh_cap = (u32)fresh_cap;
    c.status = (Status *)(slab + o_status);
    c.meta = (u32 *)(slab + o_meta);
    c.meta_cap = meta_cap;
    c.done_list = (u32 *)(slab + o_done);
    c.trace = spec.trace_cap ? (TraceRec *)(slab + o_trace) : nullptr;
    c.trace_cap = spec.trace_cap;
    c.cutoff = cutoff;
    for (int cl = 0; cl < kLeafClasses; cl++) c.class_cap[cl] = class_cap(cl);
    c.recurse = spec.skew_only ? 0 : 1;
    c.ninst = ninst;
    Counters *cnt = (Counters *)(slab + o_cnt);
    // the contexts of the two list parities (round r reads lists r & 1)
    Ctx hctx[2];
    for (int q = 0; q < 2; q++) {
      hctx[q] = c;
      for (int cl = 0; cl < kLeafClasses; cl++) {
        hctx[q].leaves_cur[cl] = (Leaf *)(slab + o_leaves[q][cl]);
        hctx[q].leaves_nxt[cl] = (Leaf *)(slab + o_leaves[q ^ 1][cl]);
      }
      hctx[q].ready_cur = (u32 *)(slab + o_ready[q]);
      hctx[q].ready_nxt = (u32 *)(slab + o_ready[q ^ 1]);
      hctx[q].fresh_cur = (u32 *)(slab + o_fresh[q]);
      hctx[q].fresh_nxt = (u32 *)(slab + o_fresh[q ^ 1]);
      hctx[q].cnt_cur = cnt + q;
      hctx[q].cnt_nxt = cnt + (q ^ 1);
    }
    Ctx *cdev = (Ctx *)(slab + P.o_ctx);

    // ---- seed the roots (host-built records)
    std::vector<Inst> hinst(ninst);
    std::vector<Node> hnodes;
    std::vector<u32> hfresh;
    std::vector<Leaf> hleaves[kLeafClasses];
    Counters hc[2];
    memset(hc, 0, sizeof(hc));
    Status hs;
    memset(&hs, 0, sizeof(hs));
    for (u32 i = 0; i < ninst; i++) {
      const InstSpec &is = spec.inst[i];
      hinst[i].keys = is.keys;
      hinst[i].vals = is.vals;
      hinst[i].dkeys = is.dkeys;
      hinst[i].dvals = is.dvals;
      hinst[i].skeys = is.skeys ? is.skeys : is.keys;
      hinst[i].svals = is.svals ? is.svals : is.vals;
      hinst[i].fkeys = is.fkeys ? is.fkeys : is.keys;
      hinst[i].fvals = is.fvals ? is.fvals : is.vals;
      hinst[i].tags = is.tags;
      hinst[i].n = is.n;
      hinst[i].cutoff = cutoff_of(i);
      hinst[i].variant = is.variant;
      if (spec.skew_only) continue;
      if (is.n == 0) {
        hs.done++;
        continue;
      }
      if (is.n <= hinst[i].cutoff) {
        int cl = 0;
        while (cl < NCLASS - 1 && is.n > class_cap(cl)) ++cl;
        Leaf L;
        L.off = 0;
        L.n = (u32)is.n;
        L.inst = i;
        L.parent = kNone;
        L.flags = KIND_ROOT | LEAF_SRC;  // from the source into A (or the final buffer)
        hleaves[cl].push_back(L);
        hc[0].leaf_elems[cl] += is.n;
      } else {
        Node nd;
        memset(&nd, 0, sizeof(nd));
        const u32 m = node_m(is.n, is.variant);
        nd.off = 0;
        nd.hash = root_hash(is.seed);
        nd.samp = kNoSamp;
        nd.n = (u32)is.n;
        nd.rows = nd.cols = nd.k = m;
        nd.inst = i;
        nd.parent = kNone;
        nd.kind = KIND_ROOT;
        nd.out = 0;
        nd.src = 1;
        const u32 id = (u32)hnodes.size();
        const u32 ncol = std::min<u32>(m, (u32)((is.n + m - 1) / m));  // non-empty columns
        const u64 last = is.n - (u64)(ncol - 1) * m;                     // the last one runs to n
        if (std::max<u64>(m, last) <= hinst[i].cutoff && m >= kHostExpandCols) {
          // a large root whose columns are leaves: spawn them here rather than
          // in one CTA of k_expand_cols
          nd.pending = (int)ncol;
          for (u32 q = 0; q < ncol; q++) {
            const u64 st0 = (u64)q * m;
            Leaf L;
            L.off = st0;
            L.n = (u32)(q + 1 == ncol ? last : (u64)m);
            L.inst = i;
            L.parent = id;
            L.flags = KIND_COL | (1u << 8) | LEAF_SRC;  // the root's columns: from the source into D
            const int cl = class_of(L.n, NCLASS);
            hleaves[cl].push_back(L);
            hc[0].leaf_elems[cl] += L.n;
          }
        } else {
          hfresh.push_back(id);
        }
        hnodes.push_back(nd);
      }
    }
    if (spec.skew_only) {
      Node nd;
      memset(&nd, 0, sizeof(nd));
      nd.n = (u32)spec.inst[0].n;
      nd.rows = (u32)spec.rows;
      nd.cols = (u32)spec.cols;
      nd.k = (u32)spec.k;
      nd.parent = kNone;
      nd.samp = kNoSamp;
      hnodes.push_back(nd);
      hc[0].ready = 1;
      hc[0].max_ready_k = nd.k;
    }
    for (int cl = 0; cl < NCLASS; cl++) hc[0].leaves[cl] = (u32)hleaves[cl].size();
    hc[0].fresh = (u32)hfresh.size();
    hs.nodes_used = (u32)hnodes.size();
    SQ_CU(cudaMemcpyAsync(c.inst, hinst.data(), sizeof(Inst) * ninst, cudaMemcpyHostToDevice, st));
    if (!hnodes.empty())
      SQ_CU(cudaMemcpyAsync(nodes, hnodes.data(), sizeof(Node) * hnodes.size(), cudaMemcpyHostToDevice, st));
    if (!hfresh.empty())
      SQ_CU(cudaMemcpyAsync(slab + o_fresh[0], hfresh.data(), 4 * hfresh.size(), cudaMemcpyHostToDevice, st));
    for (int cl = 0; cl < NCLASS; cl++)
      if (!hleaves[cl].empty())
        SQ_CU(cudaMemcpyAsync(slab + o_leaves[0][cl], hleaves[cl].data(), sizeof(Leaf) * hleaves[cl].size(),
                              cudaMemcpyHostToDevice, st));
    if (spec.skew_only) {
      const u32 zero = 0;
      SQ_CU(cudaMemcpyAsync(slab + o_ready[0], &zero, 4, cudaMemcpyHostToDevice, st));
    }
    SQ_CU(cudaMemcpyAsync(cnt, hc, sizeof(hc), cudaMemcpyHostToDevice, st));
    SQ_CU(cudaMemcpyAsync(c.status, &hs, sizeof(hs), cudaMemcpyHostToDevice, st));

    // ---- rounds
    Launcher L;
    L.st = st;
    L.prof = stats_box().profiling.load() != 0;
    SQ_CU(cudaMemcpyAsync(cdev, hctx, sizeof(hctx), cudaMemcpyHostToDevice, st));
    RoundArgs A;
    memset(&A, 0, sizeof(A));
    A.nsm = nsm;
    A.skew_only = spec.skew_only;
    A.piv_keys = spec.piv_keys;
    A.piv_vals = spec.piv_vals;
    A.bucket_start = (u64 *)spec.bucket_start;
    A.k = spec.k;
    A.skew_elems = spec.skew_only ? (double)spec.inst[0].n : 0.0;
    A.tags = 1;
    for (u32 i = 0; i < ninst; i++) A.tags &= spec.inst[i].tags != nullptr;
    u32 done = hs.done;
    int rc = 0;
    u64 rounds = 0;
    // grows the node pool so that the next round cannot overflow it
    auto grow_nodes = [&](u32 nodes_used) -> int {
      if ((u64)nodes_used + fresh_cap <= node_cap || spec.skew_only) return 0;
      const u64 ncap = std::max<u64>(2 * node_cap, (u64)nodes_used + 2 * fresh_cap);
      Node *nn = nullptr;
      SQ_CU(dalloc((void **)&nn, sizeof(Node) * ncap));
      SQ_CU(cudaMemcpyAsync(nn, nodes, sizeof(Node) * nodes_used, cudaMemcpyDeviceToDevice, st));
      SQ_CU(cudaStreamSynchronize(st));
      free_guard.rel(nodes);
      nodes = nn;
      node_cap = ncap;
      for (int q = 0; q < 2; q++) {
        hctx[q].nodes = nodes;
        hctx[q].node_cap = (u32)std::min<u64>(ncap, 0xffffffffull);
      }
      SQ_CU(cudaMemcpyAsync(cdev, hctx, sizeof(hctx), cudaMemcpyHostToDevice, st));
      return 0;
    };
    auto status_error = [&](const Status &S) -> int {
      if (!(S.error & ~ERRB_TRACE)) return 0;
      snprintf(err, errlen, "engine error bits 0x%x (1 pivot attempts, 2 nodes, 4 list, 8 arena, 16 sizes, 64 sample store)",
               S.error);
      return (S.error & ERRB_ATTEMPTS) ? 7 : ((S.error & ERRB_SIZES) ? 8 : 2);
    };
    const bool graph = spec.graph && !spec.skew_only && A.tags && !L.prof && done < ninst;
    if (graph) {
      // ---- every round on the device: one graph launch (relaunched only
      // after the host has grown the node pool)
      // every node has k = ceil(sqrt n) <= ceil(sqrt(max_n)); round up to a power of two
      int kb = 1;
      while ((1u << kb) < std::min<u64>(isqrt_ceil(max_n), max_sample() + 1)) ++kb;
      const u32 kmax = std::min<u32>(1u << kb, max_sample() + 1);
      GraphSlot &G = graph_slot(kb);
      rc = graph_prepare(G, dev, nsm, kmax, err, errlen);
      if (rc) return rc;
      struct Back {
        GraphStats gs;
        Status status;
      };
      static_assert(sizeof(Back) <= 512, "read-back buffer contract");
      void *pinned = nullptr;
      SQ_CU(pinned_readback(&pinned));
      Back &hb = *reinterpret_cast<Back *>(pinned);
      if (G.last && G.last != st) SQ_CU(cudaStreamSynchronize(G.last));  // (its launch reads G.ctx)
      G.last = st;
      if (async) {
        // enqueue the whole recursion, then the copies of its status into a
        // pending record; the scratch is freed in stream order behind them
        EngineStats per_round = G.per_round;
        PendingRun *pr = pending_take(st, (double)KEY_BYTES, per_round, ninst, err, errlen, &rc);
        if (!pr) return rc ? rc : 5;
        const Ctx pair[2] = {hctx[0], hctx[1]};
        GraphStats zero;
        memset(&zero, 0, sizeof(zero));
        SQ_CU(cudaMemcpyAsync(G.ctx, pair, sizeof(pair), cudaMemcpyHostToDevice, st));
        SQ_CU(cudaMemcpyAsync(G.gs, &zero, sizeof(zero), cudaMemcpyHostToDevice, st));
        SQ_CU(cudaGraphLaunch(G.exec, st));
        SQ_CU(cudaMemcpyAsync(&pr->gs, G.gs, sizeof(GraphStats), cudaMemcpyDeviceToHost, st));
        SQ_CU(cudaMemcpyAsync(&pr->status, c.status, sizeof(Status), cudaMemcpyDeviceToHost, st));
        return pending_commit(pr, st, err, errlen);
      }
      for (;;) {
        const int q = (int)(rounds & 1);
        const Ctx pair[2] = {hctx[q], hctx[q ^ 1]};  // the body starts with the list parity of round `rounds`
        GraphStats zero;
        memset(&zero, 0, sizeof(zero));
        SQ_CU(cudaMemcpyAsync(G.ctx, pair, sizeof(pair), cudaMemcpyHostToDevice, st));
        SQ_CU(cudaMemcpyAsync(G.gs, &zero, sizeof(zero), cudaMemcpyHostToDevice, st));
        SQ_CU(cudaGraphLaunch(G.exec, st));
        SQ_CU(cudaMemcpyAsync(&hb.gs, G.gs, sizeof(GraphStats), cudaMemcpyDeviceToHost, st));
        SQ_CU(cudaMemcpyAsync(&hb.status, c.status, sizeof(Status), cudaMemcpyDeviceToHost, st));
        SQ_CU(cudaStreamSynchronize(st));
        rounds += hb.gs.rounds;
        L.local.nodes += hb.gs.nodes;
        L.local.bytes[KF_LEAF] += 2.0 * (KEY_BYTES + 4) * (double)hb.gs.leaf_elems;
        L.local.bytes[KF_COUNT] += (KEY_BYTES + 4) * (double)hb.gs.ready_elems;
        L.local.bytes[KF_SKEW] += 2.0 * (KEY_BYTES + 4) * (double)hb.gs.ready_elems;
        for (int f = 0; f < KF_COUNT_FAMILIES; f++) L.local.launches[f] += hb.gs.rounds * G.per_round.launches[f];
        if ((rc = status_error(hb.status))) break;
        if (hb.status.done >= ninst) break;
        if (rounds >= kMaxRounds || !hb.gs.grow) {
          snprintf(err, errlen, "recursion did not finish (%llu rounds)", (unsigned long long)rounds);
          rc = 8;
          break;
        }
        if ((rc = grow_nodes(hb.status.nodes_used))) return rc;
      }
    } else {
      // ---- host-driven rounds: launches sized to the round's counts, read
      // back after every round
      struct Readback {
        Counters cnt;
        Status status;
      };
      static_assert(sizeof(Readback) <= 512, "read-back buffer contract");
      Readback *hrb = reinterpret_cast<Readback *>(spec.host_readback);
      if (!hrb) {
        void *pinned = nullptr;
        SQ_CU(pinned_readback(&pinned));
        hrb = reinterpret_cast<Readback *>(pinned);
      }
      Counters cur_cnt = hc[0];
      for (u32 r = 0;; r++) {
        if (!spec.skew_only && done >= ninst) break;
        if (spec.skew_only && r == 1) break;
        if (r >= kMaxRounds) {
          snprintf(err, errlen, "recursion did not finish");
          rc = 8;
          break;
        }
        rounds++;
        const int cur = r & 1;
        SQ_CU(issue_round(L, cdev + cur, &cur_cnt, A));
        SQ_CU(cudaMemcpyAsync(&hrb->cnt, cnt + (cur ^ 1), sizeof(Counters), cudaMemcpyDeviceToHost, st));
        SQ_CU(cudaMemcpyAsync(&hrb->status, c.status, sizeof(Status), cudaMemcpyDeviceToHost, st));
        SQ_CU(cudaStreamSynchronize(st));
        L.collect();
        if ((rc = status_error(hrb->status))) break;
        done = hrb->status.done;
        cur_cnt = hrb->cnt;
        if ((rc = grow_nodes(hrb->status.nodes_used))) return rc;
      }
    }
    if (rc == 0 && spec.trace && spec.trace_cap) {
      Status hs2;
      SQ_CU(cudaMemcpyAsync(&hs2, c.status, sizeof(Status), cudaMemcpyDeviceToHost, st));
      SQ_CU(cudaStreamSynchronize(st));
      const u32 nt = std::min(hs2.trace_used, spec.trace_cap);
      std::vector<TraceRec> tr(nt);
      if (nt)
        SQ_CU(cudaMemcpyAsync(tr.data(), c.trace, sizeof(TraceRec) * nt, cudaMemcpyDeviceToHost, st));
      SQ_CU(cudaStreamSynchronize(st));
      for (u32 i = 0; i < nt; i++) {
        spec.trace[i].off = tr[i].off;
        spec.trace[i].n = tr[i].n;
        spec.trace[i].m = tr[i].m;
        spec.trace[i].hash = tr[i].hash;
        spec.trace[i].depth = tr[i].depth;
        spec.trace[i].kind = tr[i].kind;
        spec.trace[i].attempts = tr[i].attempts;
        spec.trace[i].index = tr[i].index;
      }
      if (spec.trace_count) *spec.trace_count = hs2.trace_used;
    }
    {
      std::lock_guard<std::mutex> g(stats_box().mu);
      EngineStats &G = stats_box().s;
      for (int f = 0; f < KF_COUNT_FAMILIES; f++) {
        G.launches[f] += L.local.launches[f];
        G.ms[f] += L.local.ms[f];
        G.bytes[f] += L.local.bytes[f];
      }
      G.rounds += rounds;
      G.nodes += L.local.nodes;
      G.sorts += spec.skew_only ? 0 : ninst;
    }
    return rc;
  }

  // ---- a persistent engine that instances join between rounds ------------
  // (continuous batching).  Its lists, arena and instance slots are planned
  // once for at most total_n_cap elements and ninst_cap instances in flight;
  // admit() writes a new instance's root records into the lists of the next
  // round, step() runs one round for everything in flight and reports the
  // instances that completed in it.
  struct Session {
    SessionSpec sp;
    cudaStream_t st = nullptr;
    int nsm = 0;
    Plan P;
    char *slab = nullptr;
    Node *nodes = nullptr;
    u64 node_cap = 0;
    Ctx hctx[2];
    Ctx *cdev = nullptr;
    Counters *cnt = nullptr;
    Counters next;  // counts of the next round's lists (host copy)
    u32 nodes_used = 0, done_seen = 0;
    u64 round = 0;
    void *pinned = nullptr;

    cudaError_t dalloc(void **p, size_t bytes) {
      if (sp.dev_alloc) {
        *p = sp.dev_alloc(sp.alloc_ctx, bytes);
        return *p ? cudaSuccess : cudaErrorMemoryAllocation;
      }
      return cudaMallocAsync(p, bytes, st);
    }
    void dfree(void *p) {
      if (!p) return;
      if (sp.dev_free)
        sp.dev_free(sp.alloc_ctx, p);
      else
        cudaFreeAsync(p, st);
    }
    ~Session() {
      dfree(slab);
      dfree(nodes);
      if (pinned) cudaFreeHost(pinned);
    }

    bool has_work() const {
      if (next.ready || next.fresh) return true;
      for (int cl = 0; cl < kLeafClasses; cl++)
        if (next.leaves[cl]) return true;
      return false;
    }

    int open(const SessionSpec &spec, cudaStream_t stream, char *err, size_t errlen) {
      sp = spec;
      st = stream;
      int dev = 0;
      SQ_CU(cudaGetDevice(&dev));
      SQ_CU(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
      if (sp.cutoff_min < 2 || sp.cutoff_max > max_leaf() || sp.cutoff_min > sp.cutoff_max) {
        snprintf(err, errlen, "cutoffs [%u, %u] outside [2, %u]", sp.cutoff_min, sp.cutoff_max, max_leaf());
        return 1;
      }
      P = make_plan(sp.total_n_cap, sp.ninst_cap, sp.cutoff_min, sp.cutoff_max, 0, 0, 0, 0);
      node_cap = P.node_cap;
      SQ_CU(dalloc((void **)&slab, P.slab_bytes));
      SQ_CU(dalloc((void **)&nodes, sizeof(Node) * node_cap));
      SQ_CU(cudaMallocHost(&pinned, 512));
      Ctx c;
      memset(&c, 0, sizeof(c));
      c.inst = (Inst *)(slab + P.o_inst);
      c.nodes = nodes;
      c.node_cap = (u32)std::min<u64>(node_cap, 0xffffffffull);
      for (int cl = 0; cl < kLeafClasses; cl++) c.leaf_cap[cl] = P.leaf_cap[cl];
      c.ready_cap = (u32)P.ready_cap;
      c.wbase = (u32 *)(slab + P.o_wbase);
      c.fix = (Leaf *)(slab + P.o_fix);
      c.fix_cap = (u32)std::min<u64>(P.fix_cap, 0xffffffffull);
      c.runs = (RunCopy *)(slab + P.o_runs);
      c.runs_cap = (u32)P.runs_cap;
      c.fresh_cap = (u32)P.fresh_cap;
      c.status = (Status *)(slab + P.o_status);
      c.meta = (u32 *)(slab + P.o_meta);
      c.meta_cap = P.meta_cap;
      c.done_list = (u32 *)(slab + P.o_done);
      c.cutoff = sp.cutoff_min;
      for (int cl = 0; cl < kLeafClasses; cl++) c.class_cap[cl] = class_cap(cl);
      c.recurse = 1;
      c.ninst = sp.ninst_cap;  // also the length of the done_list ring
      cnt = (Counters *)(slab + P.o_cnt);
      for (int q = 0; q < 2; q++) {
        hctx[q] = c;
        for (int cl = 0; cl < kLeafClasses; cl++) {
          hctx[q].leaves_cur[cl] = (Leaf *)(slab + P.o_leaves[q][cl]);
          hctx[q].leaves_nxt[cl] = (Leaf *)(slab + P.o_leaves[q ^ 1][cl]);
        }
        hctx[q].ready_cur = (u32 *)(slab + P.o_ready[q]);
        hctx[q].ready_nxt = (u32 *)(slab + P.o_ready[q ^ 1]);
        hctx[q].fresh_cur = (u32 *)(slab + P.o_fresh[q]);
        hctx[q].fresh_nxt = (u32 *)(slab + P.o_fresh[q ^ 1]);
        hctx[q].cnt_cur = cnt + q;
        hctx[q].cnt_nxt = cnt + (q ^ 1);
      }
      cdev = (Ctx *)(slab + P.o_ctx);
      SQ_CU(cudaMemcpyAsync(cdev, hctx, sizeof(hctx), cudaMemcpyHostToDevice, st));
      SQ_CU(cudaMemsetAsync(cnt, 0, 2 * sizeof(Counters), st));
      SQ_CU(cudaMemsetAsync(slab + P.o_status, 0, sizeof(Status), st));
      memset(&next, 0, sizeof(next));
      SQ_CU(cudaStreamSynchronize(st));
      return 0;
    }

    int grow_nodes(u64 need, char *err, size_t errlen) {
      if (need <= node_cap) return 0;
      const u64 ncap = std::max<u64>(2 * node_cap, need + P.fresh_cap);
      Node *nn = nullptr;
      SQ_CU(dalloc((void **)&nn, sizeof(Node) * ncap));
      SQ_CU(cudaMemcpyAsync(nn, nodes, sizeof(Node) * nodes_used, cudaMemcpyDeviceToDevice, st));
      SQ_CU(cudaStreamSynchronize(st));
      dfree(nodes);
      nodes = nn;
      node_cap = ncap;
      for (int q = 0; q < 2; q++) {
        hctx[q].nodes = nodes;
        hctx[q].node_cap = (u32)std::min<u64>(ncap, 0xffffffffull);
      }
      SQ_CU(cudaMemcpyAsync(cdev, hctx, sizeof(hctx), cudaMemcpyHostToDevice, st));
      return 0;
    }

    // The instance in `slot` (free: its previous occupant completed) starts in
    // the next round.  The caller keeps the elements in flight within the plan.
    int admit(const InstSpec &is, u32 slot, char *err, size_t errlen) {
      if (slot >= sp.ninst_cap || is.n == 0 || !is.tags || is.variant) {
        snprintf(err, errlen, "bad admission (slot %u, n %llu)", slot, (unsigned long long)is.n);
        return 1;
      }
      const u64 lim = Engine::max_n();
      if (is.n > lim) {
        snprintf(err, errlen, "n = %llu exceeds the largest supported size %llu", (unsigned long long)is.n,
                 (unsigned long long)lim);
        return 1;
      }
      const u32 cut = std::min(std::max(is.cutoff ? is.cutoff : sp.cutoff_max, sp.cutoff_min), sp.cutoff_max);
      Inst hi;
      memset(&hi, 0, sizeof(hi));
      hi.keys = is.keys;
      hi.vals = is.vals;
      hi.dkeys = is.dkeys;
      hi.dvals = is.dvals;
      hi.skeys = is.skeys ? is.skeys : is.keys;
      hi.svals = is.svals ? is.svals : is.vals;
      hi.fkeys = is.fkeys ? is.fkeys : is.keys;
      hi.fvals = is.fvals ? is.fvals : is.vals;
      hi.tags = is.tags;
      hi.n = is.n;
      hi.cutoff = cut;
      hi.variant = is.variant;
      const int q = (int)(round & 1);  // the next round's lists
      std::vector<Leaf> add[kLeafClasses];
      auto put_leaf = [&](const Leaf &L) {
        const int cl = class_of(L.n, NCLASS);
        add[cl].push_back(L);
        next.leaf_elems[cl] += L.n;
      };
      Node nd;
      bool has_node = false, fresh = false;
      if (is.n <= cut) {
        Leaf L;
        L.off = 0;
        L.n = (u32)is.n;
        L.inst = slot;
        L.parent = kNone;
        L.flags = KIND_ROOT | LEAF_SRC;
        put_leaf(L);
      } else {
        if (int rc = grow_nodes((u64)nodes_used + 1 + P.fresh_cap, err, errlen)) return rc;
        memset(&nd, 0, sizeof(nd));
        const u32 m = node_m(is.n, is.variant);
        nd.off = 0;
        nd.hash = root_hash(is.seed);
        nd.samp = kNoSamp;
        nd.n = (u32)is.n;
        nd.rows = nd.cols = nd.k = m;
        nd.inst = slot;
        nd.parent = kNone;
        nd.kind = KIND_ROOT;
        nd.out = 0;
        nd.src = 1;
        has_node = true;
        const u32 id = nodes_used;
        const u32 ncol = std::min<u32>(m, (u32)((is.n + m - 1) / m));  // non-empty columns
        const u64 last = is.n - (u64)(ncol - 1) * m;                     // the last one runs to n
        if (std::max<u64>(m, last) <= cut && m >= kHostExpandCols) {     // its columns are leaves: spawn them here
          nd.pending = (int)ncol;
          for (u32 i = 0; i < ncol; i++) {
            Leaf L;
            L.off = (u64)i * m;
            L.n = (u32)(i + 1 == ncol ? last : (u64)m);
            L.inst = slot;
            L.parent = id;
            L.flags = KIND_COL | (1u << 8) | LEAF_SRC;
            put_leaf(L);
          }
        } else {
          fresh = true;
        }
      }
      for (int cl = 0; cl < NCLASS; cl++)
        if (next.leaves[cl] + add[cl].size() > P.leaf_cap[cl]) {
          snprintf(err, errlen, "leaf list %d full", cl);
          return 2;
        }
      if (fresh && next.fresh + 1 > P.fresh_cap) {
        snprintf(err, errlen, "new-node list full");
        return 2;
      }
      SQ_CU(cudaMemcpyAsync(hctx[0].inst + slot, &hi, sizeof(Inst), cudaMemcpyHostToDevice, st));
      if (has_node) {
        SQ_CU(cudaMemcpyAsync(nodes + nodes_used, &nd, sizeof(Node), cudaMemcpyHostToDevice, st));
        if (fresh) {
          const u32 id = nodes_used;
          SQ_CU(cudaMemcpyAsync(hctx[q].fresh_cur + next.fresh, &id, 4, cudaMemcpyHostToDevice, st));
          next.fresh++;
        }
        nodes_used++;
        SQ_CU(cudaMemcpyAsync(&hctx[0].status->nodes_used, &nodes_used, 4, cudaMemcpyHostToDevice, st));
      }
      for (int cl = 0; cl < NCLASS; cl++)
        if (!add[cl].empty()) {
          SQ_CU(cudaMemcpyAsync(hctx[q].leaves_cur[cl] + next.leaves[cl], add[cl].data(),
                                sizeof(Leaf) * add[cl].size(), cudaMemcpyHostToDevice, st));
          next.leaves[cl] += (u32)add[cl].size();
        }
      SQ_CU(cudaMemcpyAsync(cnt + q, &next, sizeof(Counters), cudaMemcpyHostToDevice, st));
      // pageable copies are staged before they return: the host records may go
      return 0;
    }

    // One round for everything in flight; the slots of the instances that
    // completed in it are appended to `completed`.
    int step(std::vector<u32> &completed, char *err, size_t errlen) {
      if (!has_work()) return 0;
      Launcher L;
      L.st = st;
      L.prof = stats_box().profiling.load() != 0;
      RoundArgs A;
      memset(&A, 0, sizeof(A));
      A.nsm = nsm;
      A.tags = 1;
      const int q = (int)(round & 1);
      SQ_CU(issue_round(L, cdev + q, &next, A));
      struct Readback {
        Counters cnt;
        Status status;
      };
      static_assert(sizeof(Readback) <= 512, "read-back buffer contract");
      Readback *hrb = reinterpret_cast<Readback *>(pinned);
      SQ_CU(cudaMemcpyAsync(&hrb->cnt, cnt + (q ^ 1), sizeof(Counters), cudaMemcpyDeviceToHost, st));
      SQ_CU(cudaMemcpyAsync(&hrb->status, hctx[0].status, sizeof(Status), cudaMemcpyDeviceToHost, st));
      SQ_CU(cudaStreamSynchronize(st));
      L.collect();
      const Status S = hrb->status;
      next = hrb->cnt;
      nodes_used = S.nodes_used;
      round++;
      {
        std::lock_guard<std::mutex> g(stats_box().mu);
        EngineStats &G = stats_box().s;
        for (int f = 0; f < KF_COUNT_FAMILIES; f++) {
          G.launches[f] += L.local.launches[f];
          G.ms[f] += L.local.ms[f];
          G.bytes[f] += L.local.bytes[f];
        }
        G.rounds += 1;
        G.nodes += L.local.nodes;
        G.sorts += S.done - done_seen;
      }
      if (S.error & ~ERRB_TRACE) {
        snprintf(err, errlen, "engine error bits 0x%x (1 pivot attempts, 2 nodes, 4 list, 8 arena, 16 sizes, 64 sample store)",
                 S.error);
        return (S.error & ERRB_ATTEMPTS) ? 7 : ((S.error & ERRB_SIZES) ? 8 : 2);
      }
      if (S.done != done_seen) {  // the ring of completed slots
        const u32 nd = S.done - done_seen, cap = sp.ninst_cap;
        std::vector<u32> got(nd);
        const u32 a = done_seen % cap, first = std::min(nd, cap - a);
        SQ_CU(cudaMemcpyAsync(got.data(), hctx[0].done_list + a, 4 * first, cudaMemcpyDeviceToHost, st));
        if (first < nd)
          SQ_CU(cudaMemcpyAsync(got.data() + first, hctx[0].done_list, 4 * (nd - first), cudaMemcpyDeviceToHost, st));
        SQ_CU(cudaStreamSynchronize(st));
        completed.insert(completed.end(), got.begin(), got.end());
        done_seen = S.done;
      }
      return grow_nodes((u64)nodes_used + P.fresh_cap, err, errlen);
    }
  };

  static u64 session_scratch_bytes(const SessionSpec &sp) {
    const Plan P = make_plan(sp.total_n_cap, sp.ninst_cap, sp.cutoff_min, sp.cutoff_max, 0, 0, 0, 0);
    return ((P.slab_bytes + 255) & ~(u64)255) + sizeof(Node) * P.node_cap + 4096;
  }
};


// Session entry points of one key type (expanded once per engine unit).
#define SQ_SESSION_FUNCS(SUFFIX, DTV)                                                                      \
  int session_open_##SUFFIX(const SessionSpec &sp, cudaStream_t st, void **out, char *err, size_t errlen) { \
    auto *s = new Engine<DTV>::Session();                                                                   \
    const int rc = s->open(sp, st, err, errlen);                                                            \
    if (rc) {                                                                                               \
      delete s;                                                                                             \
      return rc;                                                                                            \
    }                                                                                                       \
    *out = s;                                                                                               \
    return 0;                                                                                               \
  }                                                                                                         \
  int session_admit_##SUFFIX(void *s, const InstSpec &is, uint32_t slot, char *err, size_t errlen) {        \
    return static_cast<Engine<DTV>::Session *>(s)->admit(is, slot, err, errlen);                            \
  }                                                                                                         \
  int session_step_##SUFFIX(void *s, std::vector<uint32_t> &done, char *err, size_t errlen) {               \
    return static_cast<Engine<DTV>::Session *>(s)->step(done, err, errlen);                                 \
  }                                                                                                         \
  bool session_busy_##SUFFIX(void *s) { return static_cast<Engine<DTV>::Session *>(s)->has_work(); }       \
  void session_close_##SUFFIX(void *s) { delete static_cast<Engine<DTV>::Session *>(s); }                  \
  uint64_t session_scratch_bytes_##SUFFIX(const SessionSpec &sp) { return Engine<DTV>::session_scratch_bytes(sp); }

}  // namespace sq
