// batch_types.h — the work list of the persistent batch kernel
// (mprk_step_batch and the server), shared by the host code that builds it
// (mprk_batch.cu) and the translation unit that compiles the kernel
// (mprk_kernels.cu, through batch_kernel.cuh).
#pragma once

#include "mprk_internal.h"

namespace mprk {

struct BatchInst {
  Geom g;
  Bufs b;
  unsigned* status;  // the instance's status word
  int counter_base;  // first counter of this instance: one per stage, then completion
  int args_base;     // first entry of this instance in BatchArgs::args: one per stage
  int precision;
};

// The work items copy their stage's arguments from a table built on the
// host (stage_args of every instance and stage) in 16-byte words.
static_assert(sizeof(StageArgs) % 16 == 0, "StageArgs is copied in 16-byte words");
constexpr int ARGS_WORDS = (int)(sizeof(StageArgs) / 16);

struct BatchItem {
  int inst;
  int stage;  // 0 .. s m - 1 (s base stages per fast substep), or s m for a completion item
  int tile;   // first tile of the stage, or first chunk of the completion
  int count;  // consecutive tiles (chunks) the item covers
  int need;   // items of the previous stage this one waits for (0: none)
};

// Default tiles per work item: two in both precisions. An FP32-flux tile
// takes a few microseconds; an item's scheduling (claim, wait, argument
// copy, barriers) is mostly hidden behind the previous item, so two tiles
// per item beat four on mixed batches. mprk_batch_tune may pick others per
// size bucket.
constexpr int batch_group(int /*precision*/) { return 2; }

struct BatchArgs {
  const BatchInst* insts;
  const StageArgs* args;  // [sum over instances of s m], 16-byte aligned
  const BatchItem* items;
  int n_items;
  int* next;           // work counter
  int* counters;       // per-instance stage completion counters
  int* abort_flag;
  unsigned* status;
  long long wait_cycles;
  int withhold_inst;   // test hook: this instance's withhold_stage tiles never report done
  int withhold_stage;
};

constexpr int FIN_CHUNK = NTHREADS * 8;  // cells per completion item

// A CTA of the per-stage form: its stage arguments (an index into the
// table) and its tile of that stage, or for a completion launch the
// instance (an index into the instance table) and its chunk.
struct StageWork {
  int args;
  int tile;
};

// block size of the batch kernel per precision (the tile's own block size)
constexpr int batch_threads(int prec) { return prec == 0 ? NTHREADS : MIXED_THREADS; }

// The persistent kernel of a precision and FP64 tile rows (mprk_kernels.cu,
// the translation unit of the single-instance stage kernels, so that both
// kernels call one compiled copy of each FP64 tile body): its shared-memory
// limit and CTAs per SM, and its launch.
cudaError_t batch_prepare(int prec, int rows, size_t smem, int* per_sm);
void batch_launch(int prec, int rows, int grid, size_t smem, cudaStream_t s, const BatchArgs& A);
// The per-stage form (FP32 flux): one stage launch of `grid` CTAs of stage
// parity `parity`, and one completion launch; cudaFuncSetAttribute first
// (wave_prepare).
cudaError_t wave_prepare();
void wave_launch_stage(int parity, int grid, const StageArgs* tab, const StageWork* work, int single,
                       cudaStream_t s);
void wave_launch_finalize(int grid, const BatchInst* insts, const StageWork* work, cudaStream_t s);

}  // namespace mprk
