// Internal: the packing context (one device arena, its graphs, staging and
// last-batch state) and the two halves of a batch, shared by the C ABI
// (api.cu) and the serving loop (serve.cu).
#pragma once

#include <atomic>
#include <string>
#include <vector>

#include "tabi_internal.cuh"

namespace tabi {

// One captured launch sequence: the kernels of a batch for fan-out F with a
// row-loop CTA of `smem` dynamic bytes.  Every kernel reads the batch from
// the record at the arena's start, so the graph serves any batch.
struct GraphEntry {
  int F, smem, threads, ctas, Q, prep_group, laabb_k;  // (the progressive bound is read from the record)
  bool tail;                                           // the prefix-sum tail's kernels follow each wave
  int gutter;                                          // (selects the tail's trial kernel)
  cudaGraphExec_t exec;
};

// Launch shape of a batch: the knobs the autotuner sets.  None changes a
// result, only how the work is cut.
struct Tuning {
  int F;        // candidates per wave (scale fan-out)
  int items;    // raster warp-items per wave (sets candidates per warp)
  int threads;  // row-loop CTA: 1024 or 512 threads
  int ctas;     // row-loop CTAs per multiprocessor
  int Q;        // chart chunks per wave (lazy evaluation; 1 = all at once)
  int B;        // row loop checks the progressive area bound (1) or not (0)
};

struct TuneEntry {
  uint64_t key;  // batch class
  Tuning t;
  float ms;
};

}  // namespace tabi

struct tabi_ctx {
  int device = 0;
  char *arena = nullptr;
  size_t arena_bytes = 0;
  bool owned = false;
  std::atomic<int> busy{0};
  std::string last_error;
  int sms = 0, rowloop_dyn_max = 0, smem_per_sm = 0, smem_reserved = 0;
  cudaStream_t cap_stream = nullptr;  // stream the graphs are captured on
  std::vector<tabi::GraphEntry> graphs;
  std::vector<tabi::TuneEntry> tuned;  // autotuner results per batch class
  cudaEvent_t tev[2] = {};             // batch timing (autotuner)
  cudaEvent_t cev[2] = {};             // the overlap counter behind a batch (serving)
  // pinned host staging: the batch record going up, the results coming down
  char *hstage = nullptr;
  size_t hstage_bytes = 0;
  // the last batch, for tabi_inspect
  tabi::Pack last{};
  bool has_last = false;
  std::vector<tabi::AtlasDesc> last_desc;
  std::vector<int> last_map;  // request index -> atlas index (-1: not run)
  // optional per-stage timing (direct launches with events between stages)
  bool timing = false;
  // event pairs around the stages of one pack: prologue (3), per wave and
  // chart chunk plan, raster, compaction, row loop (4), per wave the tail
  // (1), selection
  static constexpr int kStageMarks = 4 + (4 * tabi::kMaxChunks + 1) * tabi::kScales + 4;
  cudaEvent_t ev[2 * kStageMarks] = {};
  int n_ev = 0;
  double stage_ms[8] = {};
  int64_t launches[8] = {};
  int64_t packs = 0;
};


namespace tabi {

// A batch between batch_launch and batch_finish.
struct InFlight {
  std::vector<int> order;        // request index of each atlas (largest first)
  std::vector<AtlasDesc> desc;   // the atlas table as uploaded
  Pack p{};                      // the batch record as uploaded
  size_t res_off = 0;            // results in the context's pinned staging
  std::string first_error;       // first host-check failure
  int A = 0;                     // atlases launched (0: nothing launched)
  bool timed = false;            // graph launch bracketed by tev[0..1]
  bool checked = false;          // the overlap counter ran behind the pack (cev[0..1] around it)
  size_t check_off = 0;          // its counts (3 x uint64 per atlas) in the pinned staging
};

}  // namespace tabi

tabi_status batch_launch(tabi_ctx *ctx, const tabi_params *params, tabi_request *reqs, int32_t R, void *stream,
                         bool host, const tabi::Tuning *force, tabi::Tuning *used, tabi::InFlight &fl,
                         bool check = false);
// The overlap and gutter counts (overlap, gutter, outside; -1: unchecked) of
// request r of a finished batch that ran with check = true.
void batch_quality(tabi_ctx *ctx, const tabi::InFlight &fl, int r, int64_t out[3]);
tabi_status batch_finish(tabi_ctx *ctx, tabi_request *reqs, int32_t R, tabi::InFlight &fl, float *ms_out);
