// mprk_batch.cu — many independent instances advanced together: one
// persistent launch per slow step covers every instance's stage tiles and
// step completions (mprk_step_batch).
//
// Work items (instance, stage, a run of consecutive tiles) are listed
// stage-major: all first-stage items of all instances, then all second-stage
// items, and so on, with each instance's completion items after its last
// stage. CTAs take items in list order from one atomic counter. An item of
// stage s of instance I first waits until every item of stage s-1 of I has
// finished (a per-instance counter). The tiles per item and the CTAs per SM
// come from a tuning table (mprk_batch_tune) or defaults.
// FP32-flux batches have a second form, the per-stage launches (tiles per
// item 0 in the tuning table, and the default): one launch per stage index
// over every instance that has it, and one for the step completions, in
// stream order (captured in one graph per slow step by mprk_step_batch).
// This file builds the work lists, plans and tuning; the kernel itself is
// compiled with the single-instance stage kernels (batch_kernel.cuh, included
// by mprk_kernels.cu), so that both call one compiled copy of the FP64 tile.
// Since items are taken in list order, every item an item waits on was taken
// earlier by a CTA that is already running, so the waits always end. Waits
// are bounded all the same: after a fixed number of clock cycles a CTA sets
// the status word's timeout bit and an abort flag, and every CTA then drains
// without touching the states (no trap, no hang).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <sstream>
#include <mutex>
#include <string>
#include <vector>

#include "batch_types.h"
#include "mprk.h"
#include "mprk_internal.h"


using namespace mprk;

// ---------------------------------------------------------------------------
// Host side: a plan per set of instances (cached), captured in a CUDA graph.
// ---------------------------------------------------------------------------
namespace {

// What the per-stage form launches from: the work lists and their bounds,
// and for the launches over a single instance (single[g][k] >= 0: its stage
// argument index) the host copies of the arguments and tensor maps. Those
// launches take the single-instance FP32-flux kernel (launch_stage):
// arguments as kernel parameters and tensor-copied tiles, the code mprk_step
// runs, so that an instance alone in a launch steps exactly as it would
// alone, and as fast.
struct WaveLaunches {
  std::vector<std::vector<int>> off, single;
  std::vector<StageArgs> h_args;  // the argument table (host copy)
  std::vector<int> args_inst;     // instance of each argument entry
  std::vector<StageMaps> h_maps;  // per instance
};

// Streams and events for the groups of the per-stage form beyond the first
// (which runs on the batch's own stream).
struct WaveStreams {
  std::vector<cudaStream_t> aux;
  std::vector<cudaEvent_t> ev;  // [0] the fork, [g] group g's join
  cudaError_t ensure(int groups) {
    while ((int)aux.size() < groups - 1) {
      cudaStream_t st;
      cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
      if (e != cudaSuccess) return e;
      aux.push_back(st);
    }
    while ((int)ev.size() < groups) {
      cudaEvent_t e0;
      cudaError_t e = cudaEventCreateWithFlags(&e0, cudaEventDisableTiming);
      if (e != cudaSuccess) return e;
      ev.push_back(e0);
    }
    return cudaSuccess;
  }
  void release() {
    for (cudaStream_t st : aux) {
      cudaStreamSynchronize(st);
      cudaStreamDestroy(st);
    }
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
    aux.clear();
    ev.clear();
  }
};

struct Plan {
  std::vector<const void*> key;
  int precision = 0;
  int bucket = 0;      // size bucket of the instance set (tuning key)
  int group = 0;       // tiles per work item
  int rows = TZ;       // FP64 tile rows (TZ, or TZ / 2 with two threads per cell)
  int per_sm = 0;      // CTAs per SM of the persistent launch
  int per_sm_req = 0;  // CTAs per SM asked for (0: as many as fit)
  int n_items = 0;
  int n_counters = 0;
  int grid = 0;
  long long cell_stages = 0;
  BatchInst* d_insts = nullptr;
  StageArgs* d_args = nullptr;
  BatchItem* d_items = nullptr;
  int* d_ctr = nullptr;  // [0] next, [1] abort, [2..] counters
  int form = 0;                   // 0 persistent launch, 1 per-stage launches
  StageWork* d_work = nullptr;    // per-stage form: the launches' work lists
  WaveLaunches wl;                 // per-stage form: launch bounds and host tables
  WaveStreams ws;                 // the groups' streams (per-stage form)
  cudaGraphExec_t exec = nullptr;
  cudaStream_t stream = nullptr;
  long long wait_cycles = 0;
  int withhold_inst = -1, withhold_stage = -1;
};

std::mutex g_batch_mu;
std::vector<Plan*> g_plans;

// ---- launch tuning ---------------------------------------------------------
// Two choices of the persistent launch change no result: the tiles per work
// item and the CTAs per SM. The table holds, per precision and size bucket
// (floor(log2) of the mean cells per instance), the fastest pair
// mprk_batch_tune measured, with the name of the GPU it ran on. Plans
// without an entry take the defaults (batch_group tiles, every CTA that fits).
// Tiles per item 0 stands for the per-stage form of FP32-flux batches; its
// CTAs per SM field then holds the number of instance groups (0: two).
struct TuneVal {
  int group, per_sm;
  double ms;
  int rows;  // FP64 tile rows of the batch kernel (the FP32-flux tile is fixed)
};
std::mutex g_tune_mu;
std::map<std::pair<int, int>, TuneVal> g_tune;
std::string g_tune_gpu;
// Tile shapes of single-instance FP64 stage launches per size bucket (floor
// log2 of the launch's cells), measured by mprk_tile_tune.
struct ShapeVal {
  TileShape shape;
  double ms;
};
std::map<int, ShapeVal> g_shape;

int size_bucket(const std::vector<BatchInst>& hinst) {
  double cells = 0;
  for (const BatchInst& bi : hinst) cells += (double)bi.g.nx * bi.g.nz;
  const double mean = hinst.empty() ? 1.0 : cells / hinst.size();
  return std::max(0, std::min(40, (int)std::floor(std::log2(std::max(mean, 1.0)))));
}

// The tuned (group, per_sm, FP64 tile rows) of a precision and bucket, or
// the defaults (per_sm 0: as many as fit; TZ rows).
void tuned_choice(int prec, int bucket, int* group, int* per_sm, int* rows) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tune.find({prec, bucket});
  if (it != g_tune.end()) {
    *group = it->second.group;
    *per_sm = it->second.per_sm;
    *rows = prec == 0 ? it->second.rows : MTZ;
  } else {
    *group = prec == 0 ? batch_group(prec) : 0;
    *per_sm = 0;
    *rows = prec == 0 ? TZ : MTZ;
  }
}

int cells_bucket(double cells) { return std::max(0, std::min(40, (int)std::floor(std::log2(std::max(cells, 1.0))))); }

std::string device_name() {
  int dev = 0;
  cudaDeviceProp prop;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
    cudaGetLastError();
    return "";
  }
  return prop.name;
}

int bfail(int code, const std::string& msg) {
  set_last_error(msg);
  return code;
}

void free_plan(Plan* p) {
  if (!p) return;
  if (p->exec) cudaGraphExecDestroy(p->exec);
  cudaFree(p->d_insts);
  cudaFree(p->d_args);
  cudaFree(p->d_items);
  cudaFree(p->d_ctr);
  cudaFree(p->d_work);
  p->ws.release();
  delete p;
}

}  // namespace


namespace {

// Stage arguments of an instance of the batch: FP64 tiles of `rows` rows.
StageArgs batch_stage_args(const BatchInst& bi, int st, int rows) {
  StageArgs a = stage_args(bi.g, bi.b, st);
  if (bi.precision == 0) a.tz = rows;
  return a;
}

// The stage arguments of every instance and stage, in instance order; sets
// each instance's args_base.
void args_table(std::vector<BatchInst>& hinst, int rows, std::vector<StageArgs>& out) {
  out.clear();
  for (BatchInst& bi : hinst) {
    bi.args_base = (int)out.size();
    for (int st = 0; st < bi.g.s * bi.g.m; st++) out.push_back(batch_stage_args(bi, st, rows));
  }
}

// The stage-major work list: all first-stage items of all instances, then
// all second-stage items, ...; each instance's completion items follow its
// last stage. Items group G consecutive tiles.
void build_items(const std::vector<BatchInst>& hinst, int G, int rows, std::vector<BatchItem>& items,
                 long long* cell_stages) {
  int max_stages = 0;
  for (const BatchInst& bi : hinst) max_stages = std::max(max_stages, bi.g.s * bi.g.m);
  long long cs = 0;
  items.clear();
  for (int st = 0; st <= max_stages; st++) {
    for (int j = 0; j < (int)hinst.size(); j++) {
      const Geom& g = hinst[j].g;
      const int ms = g.s * g.m;  // s stages per fast substep
      if (st > ms) continue;
      auto ntiles = [&](int s) {
        if (s < ms) return stage_tiles(batch_stage_args(hinst[j], s, rows));
        const int rows = ((g.m & 1) || hinst[j].b.dA) ? g.nz : g.n1_r;  // as finalize_chunk
        const long long total = 4LL * rows * g.nx;
        return (int)((total + FIN_CHUNK - 1) / FIN_CHUNK);
      };
      const int nt = ntiles(st);
      const int need = st == 0 ? 0 : (ntiles(st - 1) + G - 1) / G;
      for (int t = 0; t < nt; t += G) items.push_back({j, st, t, std::min(G, nt - t), need});
      if (st < ms) cs += (long long)(g.nz - stage_args(g, hinst[j].b, st).row0) * g.nx;
    }
  }
  *cell_stages = cs;
}

// The work lists of the per-stage form. The instances are split into
// `groups` groups of about equal work (largest first, each to the least
// loaded group); each group's launches go on a stream of their own, so that
// one group's launch tail overlaps another group's work. Launch s of a group
// (s = 0 .. the most stages of its instances, minus one) lists the (stage
// argument index, tile) pairs of its instances that have a stage s, and a
// last launch the (instance, chunk) pairs of their step completions. Launch
// s of group g takes the entries off[g][s] .. off[g][s+1] (a completion
// entry holds the instance and 4 r0 + c: the band of rows from r0 of
// component c). Needs the
// args_base of args_table.
void build_wave(const std::vector<BatchInst>& hinst, int groups, std::vector<StageWork>& work,
                std::vector<std::vector<int>>& off, std::vector<std::vector<int>>& single,
                long long* cell_stages) {
  const int n = (int)hinst.size();
  groups = std::max(1, std::min(groups, n));
  auto step_cs = [&](int j) {
    long long cs = 0;
    for (int st = 0; st < hinst[j].g.s * hinst[j].g.m; st++)
      cs += (long long)(hinst[j].g.nz - batch_stage_args(hinst[j], st, MTZ).row0) * hinst[j].g.nx;
    return cs;
  };
  std::vector<int> order(n);
  std::vector<long long> cs(n);
  for (int j = 0; j < n; j++) {
    order[j] = j;
    cs[j] = step_cs(j);
  }
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cs[x] > cs[y]; });
  std::vector<std::vector<int>> members(groups);
  std::vector<long long> load(groups, 0);
  for (int j : order) {
    const int g = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    members[g].push_back(j);
    load[g] += cs[j];
  }
  long long total = 0;
  work.clear();
  off.assign(groups, std::vector<int>());
  single.assign(groups, std::vector<int>());
  for (int g = 0; g < groups; g++) {
    std::sort(members[g].begin(), members[g].end());  // instance order within a launch
    int max_stages = 0;
    for (int j : members[g]) max_stages = std::max(max_stages, hinst[j].g.s * hinst[j].g.m);
    off[g].push_back((int)work.size());
    for (int st = 0; st < max_stages; st++) {
      int n_in = 0, only = -1;
      for (int j : members[g]) {
        const BatchInst& bi = hinst[j];
        if (st >= bi.g.s * bi.g.m) continue;
        const int nt = stage_tiles(batch_stage_args(bi, st, MTZ));
        for (int t = 0; t < nt; t++) work.push_back({bi.args_base + st, t});
        n_in++;
        only = bi.args_base + st;
      }
      off[g].push_back((int)work.size());
      single[g].push_back(n_in == 1 ? only : -1);  // a launch over one instance reads no work list
    }
    for (int j : members[g]) {
      // bands of rows of one component (finalize_rows in batch_kernel.cuh)
      const Geom& gm = hinst[j].g;
      const int rows = ((gm.m & 1) || hinst[j].b.dA) ? gm.nz : gm.n1_r;
      const int band = std::max(1, FIN_CHUNK / gm.nx);
      for (int c = 0; c < 4; c++)
        for (int r0 = 0; r0 < rows; r0 += band) work.push_back({j, 4 * r0 + c});
      total += cs[j];
    }
    off[g].push_back((int)work.size());
  }
  *cell_stages = total;
}

// The host copies of the argument table and each instance's tensor maps.
cudaError_t wave_host_tables(const std::vector<BatchInst>& hinst, const std::vector<StageArgs>& hargs,
                             WaveLaunches& L) {
  L.h_args = hargs;
  L.args_inst.assign(hargs.size(), 0);
  L.h_maps.assign(hinst.size(), StageMaps{});
  for (size_t j = 0; j < hinst.size(); j++) {
    for (int st = 0; st < hinst[j].g.s * hinst[j].g.m; st++) {
      L.args_inst[hinst[j].args_base + st] = (int)j;
      L.h_args[hinst[j].args_base + st].status = hinst[j].status;
    }
    cudaError_t e = make_stage_maps(hinst[j].g, hinst[j].b, &L.h_maps[j]);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Launches of one slow step in the per-stage form: group 0 on stream s, the
// others forked from s onto their own streams and joined back into s.
void wave_step(const WaveLaunches& L, const BatchInst* d_insts, const StageArgs* d_args, const StageWork* d_work,
               cudaStream_t s, WaveStreams& ws) {
  const std::vector<std::vector<int>>& off = L.off;
  const int groups = (int)off.size();
  if (groups > 1) {
    cudaEventRecord(ws.ev[0], s);
    for (int g = 1; g < groups; g++) cudaStreamWaitEvent(ws.aux[g - 1], ws.ev[0], 0);
  }
  for (int g = 0; g < groups; g++) {
    const cudaStream_t st = g == 0 ? s : ws.aux[g - 1];
    const std::vector<int>& o = off[g];
    const int launches = (int)o.size() - 1;
    for (int k = 0; k + 1 < launches; k++) {
      const int one = L.single[g][k];
      if (one >= 0)
        launch_stage(L.h_args[one], 1, o[k + 1] - o[k], st, &L.h_maps[L.args_inst[one]]);
      else
        wave_launch_stage(k & 1, o[k + 1] - o[k], d_args, d_work + o[k], -1, st);
    }
    wave_launch_finalize(o[launches] - o[launches - 1], d_insts, d_work + o[launches - 1], st);
  }
  for (int g = 1; g < groups; g++) {
    cudaEventRecord(ws.ev[g], ws.aux[g - 1]);
    cudaStreamWaitEvent(s, ws.ev[g], 0);
  }
}

// Instance groups of the per-stage form: the tuned count (the table's CTAs
// per SM field holds it for this form), else two.
constexpr int WAVE_GROUPS_DEFAULT = 2;
int wave_groups(int want) { return want > 0 ? want : WAVE_GROUPS_DEFAULT; }

// The form of a batch: 1 (per-stage launches) for FP32-flux batches with
// tiles per item 0, else 0 (the persistent launch).
int batch_form(int precision, int group) { return precision == 1 && group == 0 ? 1 : 0; }

// group / per_sm / rows: the launch choices (group 0: the per-stage form of
// FP32 flux), or group < 0 for the tuned (else default) ones.
int build_plan(mprk_instance* const* insts, int count, long long wait_cycles, int wi, int ws,
               cudaStream_t stream, int group, int per_sm_want, int rows, Plan** out) {
  Plan* p = new Plan();
  p->wait_cycles = wait_cycles;
  p->withhold_inst = wi;
  p->withhold_stage = ws;
  std::vector<BatchInst> hinst(count);
  unsigned* status = nullptr;
  for (int j = 0; j < count; j++) {
    cudaStream_t s;
    unsigned* st;
    int prec;
    int rc = instance_view(insts[j], &hinst[j].g, &hinst[j].b, &prec, &s, &st);
    if (rc) { free_plan(p); return rc; }
    if (hinst[j].g.ny > 1) {
      free_plan(p);
      return bfail(MPRK_EINVAL, "batches take 2-D instances");
    }
    hinst[j].status = st;
    if (j == 0) {
      p->precision = prec;
      p->stream = stream ? stream : s;
      status = st;
    } else if (prec != p->precision) {
      free_plan(p);
      return bfail(MPRK_EINVAL, "all instances of a batch need the same precision");
    }
    hinst[j].precision = prec;
    hinst[j].counter_base = p->n_counters;
    p->n_counters += hinst[j].g.s * hinst[j].g.m + 1;
    p->key.push_back(insts[j]);
  }
  p->bucket = size_bucket(hinst);
  if (group < 0) tuned_choice(p->precision, p->bucket, &group, &per_sm_want, &rows);
  // FP64 has no per-stage form, and the test hook withholds a persistent
  // launch's completion reports
  if (group == 0 && (p->precision == 0 || wi >= 0)) group = batch_group(p->precision);
  if (p->precision != 0) rows = MTZ;
  else if (rows != TZ && rows != TZ / 2) rows = TZ;
  p->group = group;
  p->rows = rows;
  p->per_sm_req = per_sm_want;
  std::vector<StageArgs> hargs;
  args_table(hinst, rows, hargs);
  cudaError_t e;
  p->form = batch_form(p->precision, group);
  if (p->form == 1) {
    std::vector<StageWork> work;
    build_wave(hinst, wave_groups(per_sm_want), work, p->wl.off, p->wl.single, &p->cell_stages);
    if ((e = wave_host_tables(hinst, hargs, p->wl)) != cudaSuccess) {
      free_plan(p);
      return bfail(MPRK_ECUDA, std::string("batch plan tensor maps: ") + cudaGetErrorString(e));
    }
    if ((e = cudaMalloc(&p->d_insts, sizeof(BatchInst) * count)) != cudaSuccess ||
        (e = cudaMalloc(&p->d_args, sizeof(StageArgs) * hargs.size())) != cudaSuccess ||
        (e = cudaMalloc(&p->d_work, sizeof(StageWork) * work.size())) != cudaSuccess) {
      free_plan(p);
      return bfail(MPRK_ENOMEM, std::string("batch plan allocation: ") + cudaGetErrorString(e));
    }
    if ((e = cudaMemcpy(p->d_insts, hinst.data(), sizeof(BatchInst) * count, cudaMemcpyHostToDevice)) !=
            cudaSuccess ||
        (e = cudaMemcpy(p->d_args, hargs.data(), sizeof(StageArgs) * hargs.size(), cudaMemcpyHostToDevice)) !=
            cudaSuccess ||
        (e = cudaMemcpy(p->d_work, work.data(), sizeof(StageWork) * work.size(), cudaMemcpyHostToDevice)) !=
            cudaSuccess ||
        (e = wave_prepare()) != cudaSuccess || (e = p->ws.ensure((int)p->wl.off.size())) != cudaSuccess) {
      free_plan(p);
      return bfail(MPRK_ECUDA, std::string("batch plan upload: ") + cudaGetErrorString(e));
    }
    cudaGraph_t graph = nullptr;
    e = cudaStreamBeginCapture(p->stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      wave_step(p->wl, p->d_insts, p->d_args, p->d_work, p->stream, p->ws);
      cudaError_t el = cudaGetLastError();
      e = cudaStreamEndCapture(p->stream, &graph);
      if (el != cudaSuccess) e = el;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&p->exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      free_plan(p);
      return bfail(MPRK_ECUDA, std::string("batch graph: ") + cudaGetErrorString(e));
    }
    *out = p;
    return MPRK_OK;
  }
  std::vector<BatchItem> items;
  build_items(hinst, group, rows, items, &p->cell_stages);
  p->n_items = (int)items.size();
  if ((e = cudaMalloc(&p->d_insts, sizeof(BatchInst) * count)) != cudaSuccess ||
      (e = cudaMalloc(&p->d_args, sizeof(StageArgs) * hargs.size())) != cudaSuccess ||
      (e = cudaMalloc(&p->d_items, sizeof(BatchItem) * items.size())) != cudaSuccess ||
      (e = cudaMalloc(&p->d_ctr, sizeof(int) * (2 + p->n_counters))) != cudaSuccess) {
    free_plan(p);
    return bfail(MPRK_ENOMEM, std::string("batch plan allocation: ") + cudaGetErrorString(e));
  }
  if (reinterpret_cast<uintptr_t>(p->d_args) % 16 != 0) {
    free_plan(p);
    return bfail(MPRK_ECUDA, "batch plan: argument table not 16-byte aligned");
  }
  if ((e = cudaMemcpy(p->d_insts, hinst.data(), sizeof(BatchInst) * count, cudaMemcpyHostToDevice)) !=
          cudaSuccess ||
      (e = cudaMemcpy(p->d_args, hargs.data(), sizeof(StageArgs) * hargs.size(), cudaMemcpyHostToDevice)) !=
          cudaSuccess ||
      (e = cudaMemcpy(p->d_items, items.data(), sizeof(BatchItem) * items.size(), cudaMemcpyHostToDevice)) !=
          cudaSuccess) {
    free_plan(p);
    return bfail(MPRK_ECUDA, std::string("batch plan upload: ") + cudaGetErrorString(e));
  }
  // grid: every CTA resident (persistent kernel)
  const size_t smem = stage_smem_bytes(p->precision);
  int per_sm = 0, dev = 0, sms = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
      (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) {
    free_plan(p);
    return bfail(MPRK_ECUDA, std::string("batch plan device query: ") + cudaGetErrorString(e));
  }
  // dynamic shared memory above 48 KB needs the kernel attribute first
  e = batch_prepare(p->precision, p->rows, smem, &per_sm);
  if (e != cudaSuccess || per_sm < 1) {
    free_plan(p);
    return bfail(MPRK_ECUDA, std::string("occupancy query: ") + cudaGetErrorString(e) + ", " +
                                 std::to_string(per_sm) + " blocks per SM");
  }
  p->per_sm_req = per_sm_want;
  if (per_sm_want > 0) per_sm = std::min(per_sm, per_sm_want);
  p->per_sm = per_sm;
  p->grid = std::min(per_sm * sms, p->n_items);
  // capture: reset the counters, then the persistent launch
  BatchArgs A;
  A.insts = p->d_insts;
  A.args = p->d_args;
  A.items = p->d_items;
  A.n_items = p->n_items;
  A.next = p->d_ctr;
  A.abort_flag = p->d_ctr + 1;
  A.counters = p->d_ctr + 2;
  A.status = status;
  A.wait_cycles = p->wait_cycles;
  A.withhold_inst = p->withhold_inst;
  A.withhold_stage = p->withhold_stage;
  cudaGraph_t graph = nullptr;
  e = cudaStreamBeginCapture(p->stream, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaMemsetAsync(p->d_ctr, 0, sizeof(int) * (2 + p->n_counters), p->stream);
    batch_launch(p->precision, p->rows, p->grid, smem, p->stream, A);
    cudaError_t el = cudaGetLastError();
    e = cudaStreamEndCapture(p->stream, &graph);
    if (el != cudaSuccess) e = el;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&p->exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    free_plan(p);
    return bfail(MPRK_ECUDA, std::string("batch graph: ") + cudaGetErrorString(e));
  }
  *out = p;
  return MPRK_OK;
}

// A cached plan for this instance set whose launch choice is still the
// tuned one (a plan built before a tuning run is rebuilt).
Plan* find_plan(mprk_instance* const* insts, int count, long long wait_cycles, int wi, int ws,
                cudaStream_t stream) {
  for (size_t k = 0; k < g_plans.size(); k++) {
    Plan* p = g_plans[k];
    if ((int)p->key.size() != count || p->wait_cycles != wait_cycles || p->withhold_inst != wi ||
        p->withhold_stage != ws || (stream && p->stream != stream))
      continue;
    bool same = true;
    for (int j = 0; j < count && same; j++) same = p->key[j] == insts[j];
    if (!same) continue;
    int group, per_sm, rows;
    tuned_choice(p->precision, p->bucket, &group, &per_sm, &rows);
    if (group == p->group && per_sm == p->per_sm_req && rows == p->rows) return p;
    if (p->stream) cudaStreamSynchronize(p->stream);
    free_plan(p);
    g_plans.erase(g_plans.begin() + k);
    return nullptr;
  }
  return nullptr;
}

// Every member non-null and listed once: two work items on one instance's
// buffers in the same launch would race.
int check_members(mprk_instance* const* insts, int count) {
  std::vector<const void*> v(insts, insts + count);
  for (const void* p : v)
    if (!p) return bfail(MPRK_EINVAL, "NULL instance in batch");
  std::sort(v.begin(), v.end());
  if (std::adjacent_find(v.begin(), v.end()) != v.end())
    return bfail(MPRK_EINVAL, "an instance appears twice in the batch");
  return MPRK_OK;
}

int step_batch(mprk_instance* const* insts, int count, int n, long long wait_cycles, int wi, int ws,
               cudaStream_t stream, long long* cell_stages) {
  if (!insts || count <= 0) return bfail(MPRK_EINVAL, "empty batch");
  if (n < 0) return bfail(MPRK_EINVAL, "negative step count");
  if (int rc = check_members(insts, count)) return rc;
  std::lock_guard<std::mutex> lk(g_batch_mu);
  Plan* p = find_plan(insts, count, wait_cycles, wi, ws, stream);
  if (!p) {
    int rc = build_plan(insts, count, wait_cycles, wi, ws, stream, -1, 0, 0, &p);
    if (rc) return rc;
    if (g_plans.size() >= 64) {
      // the oldest plan's launches may still be running on its stream
      Plan* old = g_plans.front();
      if (old->stream) cudaStreamSynchronize(old->stream);
      free_plan(old);
      g_plans.erase(g_plans.begin());
    }
    g_plans.push_back(p);
  }
  if (cell_stages) *cell_stages = p->cell_stages;
  // order: the batch stream waits for every instance's queued work, and every
  // instance stream waits for the batch before its own later work
  std::vector<cudaStream_t> others;
  for (int j = 0; j < count; j++) {
    cudaStream_t s = instance_stream(insts[j]);
    if (s != p->stream && std::find(others.begin(), others.end(), s) == others.end()) others.push_back(s);
  }
  cudaEvent_t ev = nullptr;
  if (!others.empty()) {
    cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return bfail(MPRK_ECUDA, std::string("event: ") + cudaGetErrorString(e));
    for (cudaStream_t s : others) {
      cudaEventRecord(ev, s);
      cudaStreamWaitEvent(p->stream, ev, 0);
    }
  }
  for (int s = 0; s < n; s++) {
    cudaError_t e = cudaGraphLaunch(p->exec, p->stream);
    if (e != cudaSuccess) {
      if (ev) cudaEventDestroy(ev);
      return bfail(MPRK_ECUDA, std::string("batch launch: ") + cudaGetErrorString(e));
    }
  }
  if (ev) {
    cudaEventRecord(ev, p->stream);
    for (cudaStream_t s : others) cudaStreamWaitEvent(s, ev, 0);
    cudaEventDestroy(ev);
  }
  for (int j = 0; j < count; j++) instance_count_steps(insts[j], n);
  return MPRK_OK;
}

}  // namespace

namespace mprk {

// ---------------------------------------------------------------------------
// BatchRunner: the same persistent launch without a graph, for a resident set
// that changes between slow steps (the server). The work list is rebuilt and
// uploaded only when the set changes; device buffers grow stream-ordered.
// ---------------------------------------------------------------------------
struct BatchRunner {
  int precision = 0;
  cudaStream_t stream = nullptr;
  std::vector<const void*> key;
  BatchInst* d_insts = nullptr;
  StageArgs* d_args = nullptr;
  BatchItem* d_items = nullptr;
  int* d_ctr = nullptr;
  size_t cap_insts = 0, cap_args = 0, cap_items = 0, cap_ctr = 0;
  int n_items = 0, n_counters = 0, grid = 0, per_sm = 0, sms = 0;
  int rows = TZ;  // FP64 tile rows of the current work list
  long long cell_stages = 0;
  unsigned* status = nullptr;
  int form = 0;  // as Plan::form
  StageWork* d_work = nullptr;
  size_t cap_work = 0;
  WaveLaunches wl;
  WaveStreams ws;
};

BatchRunner* runner_create(int precision, cudaStream_t stream) {
  BatchRunner* r = new BatchRunner();
  r->precision = precision;
  r->stream = stream;
  return r;
}

void runner_destroy(BatchRunner* r) {
  if (!r) return;
  if (r->d_insts) cudaFreeAsync(r->d_insts, r->stream);
  if (r->d_args) cudaFreeAsync(r->d_args, r->stream);
  if (r->d_items) cudaFreeAsync(r->d_items, r->stream);
  if (r->d_ctr) cudaFreeAsync(r->d_ctr, r->stream);
  if (r->d_work) cudaFreeAsync(r->d_work, r->stream);
  r->ws.release();
  delete r;
}

template <typename T>
static cudaError_t grow(T** p, size_t* cap, size_t need, cudaStream_t s) {
  if (need <= *cap) return cudaSuccess;
  size_t c = std::max(need, *cap * 2);
  if (*p) cudaFreeAsync(*p, s);
  *p = nullptr;
  *cap = 0;
  cudaError_t e = cudaMallocAsync((void**)p, c * sizeof(T), s);
  if (e == cudaSuccess) *cap = c;
  return e;
}

void runner_invalidate(BatchRunner* r) {
  if (r) r->key.clear();
}

int runner_step(BatchRunner* r, mprk_instance* const* insts, int count, long long* cell_stages) {
  if (count <= 0) return MPRK_OK;
  bool same = (int)r->key.size() == count;
  for (int j = 0; j < count && same; j++) same = r->key[j] == insts[j];
  if (!same) {
    // forget the previous set first: a failure below may already have
    // replaced its device buffers, and must make the next call rebuild
    r->key.clear();
    std::vector<BatchInst> hinst(count);
    int n_counters = 0;
    for (int j = 0; j < count; j++) {
      cudaStream_t s;
      unsigned* st;
      int prec;
      int rc = instance_view(insts[j], &hinst[j].g, &hinst[j].b, &prec, &s, &st);
      if (rc) return rc;
      if (prec != r->precision) return bfail(MPRK_EINVAL, "batch runner: precision mismatch");
      if (hinst[j].g.ny > 1) return bfail(MPRK_EINVAL, "batch runner: 2-D instances only");
      hinst[j].status = st;
      hinst[j].precision = prec;
      hinst[j].counter_base = n_counters;
      n_counters += hinst[j].g.s * hinst[j].g.m + 1;
      if (j == 0) r->status = st;
    }
    int group, per_sm_want, rows;
    tuned_choice(r->precision, size_bucket(hinst), &group, &per_sm_want, &rows);
    r->form = batch_form(r->precision, group);
    cudaError_t e;
    if (r->form == 1) {
      std::vector<StageArgs> hargs;
      args_table(hinst, MTZ, hargs);
      std::vector<StageWork> work;
      long long cs = 0;
      build_wave(hinst, wave_groups(per_sm_want), work, r->wl.off, r->wl.single, &cs);
      if ((e = wave_host_tables(hinst, hargs, r->wl)) != cudaSuccess)
        return bfail(MPRK_ECUDA, std::string("batch runner tensor maps: ") + cudaGetErrorString(e));
      e = grow(&r->d_insts, &r->cap_insts, (size_t)count, r->stream);
      if (e == cudaSuccess) e = grow(&r->d_args, &r->cap_args, hargs.size(), r->stream);
      if (e == cudaSuccess) e = grow(&r->d_work, &r->cap_work, work.size(), r->stream);
      if (e != cudaSuccess) return bfail(MPRK_ENOMEM, std::string("batch runner: ") + cudaGetErrorString(e));
      // pageable sources: the copies are staged before the calls return
      e = cudaMemcpyAsync(r->d_insts, hinst.data(), sizeof(BatchInst) * count, cudaMemcpyHostToDevice,
                          r->stream);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(r->d_args, hargs.data(), sizeof(StageArgs) * hargs.size(), cudaMemcpyHostToDevice,
                            r->stream);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(r->d_work, work.data(), sizeof(StageWork) * work.size(), cudaMemcpyHostToDevice,
                            r->stream);
      if (e == cudaSuccess) e = wave_prepare();
      if (e == cudaSuccess) e = r->ws.ensure((int)r->wl.off.size());
      if (e != cudaSuccess) return bfail(MPRK_ECUDA, std::string("batch runner upload: ") + cudaGetErrorString(e));
      r->key.assign(insts, insts + count);
      r->cell_stages = cs;
    } else {
      if (r->precision == 0 && rows != r->rows) r->per_sm = 0;  // another kernel: query its occupancy
      r->rows = rows;
      std::vector<StageArgs> hargs;
      args_table(hinst, rows, hargs);
      std::vector<BatchItem> items;
      long long cs = 0;
      build_items(hinst, group, rows, items, &cs);
      e = grow(&r->d_insts, &r->cap_insts, (size_t)count, r->stream);
      if (e == cudaSuccess) e = grow(&r->d_args, &r->cap_args, hargs.size(), r->stream);
      if (e == cudaSuccess) e = grow(&r->d_items, &r->cap_items, items.size(), r->stream);
      if (e == cudaSuccess) e = grow(&r->d_ctr, &r->cap_ctr, (size_t)(2 + n_counters), r->stream);
      if (e != cudaSuccess) return bfail(MPRK_ENOMEM, std::string("batch runner: ") + cudaGetErrorString(e));
      // pageable sources: the copies are staged before the calls return
      if (reinterpret_cast<uintptr_t>(r->d_args) % 16 != 0)
        return bfail(MPRK_ECUDA, "batch runner: argument table not 16-byte aligned");
      e = cudaMemcpyAsync(r->d_insts, hinst.data(), sizeof(BatchInst) * count, cudaMemcpyHostToDevice,
                          r->stream);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(r->d_args, hargs.data(), sizeof(StageArgs) * hargs.size(), cudaMemcpyHostToDevice,
                            r->stream);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(r->d_items, items.data(), sizeof(BatchItem) * items.size(), cudaMemcpyHostToDevice,
                            r->stream);
      if (e != cudaSuccess) return bfail(MPRK_ECUDA, std::string("batch runner upload: ") + cudaGetErrorString(e));
      r->key.assign(insts, insts + count);
      r->n_items = (int)items.size();
      r->n_counters = n_counters;
      r->cell_stages = cs;
      if (r->per_sm == 0) {
        const size_t smem = stage_smem_bytes(r->precision);
        int dev = 0;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
            (e = cudaDeviceGetAttribute(&r->sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) {
          r->key.clear();  // rebuild on the next call
          return bfail(MPRK_ECUDA, std::string("batch runner device query: ") + cudaGetErrorString(e));
        }
        e = batch_prepare(r->precision, r->rows, smem, &r->per_sm);
        if (e != cudaSuccess || r->per_sm < 1) {
          r->key.clear();
          r->per_sm = 0;
          return bfail(MPRK_ECUDA, "batch runner: occupancy query failed");
        }
      }
      r->grid = (per_sm_want > 0 ? std::min(per_sm_want, r->per_sm) : r->per_sm) * r->sms;
    }
  }
  cudaError_t e;
  if (r->form == 1) {
    wave_step(r->wl, r->d_insts, r->d_args, r->d_work, r->stream, r->ws);
  } else {
    BatchArgs A;
    A.insts = r->d_insts;
    A.args = r->d_args;
    A.items = r->d_items;
    A.n_items = r->n_items;
    A.next = r->d_ctr;
    A.abort_flag = r->d_ctr + 1;
    A.counters = r->d_ctr + 2;
    A.status = r->status;
    A.wait_cycles = 2000000000LL;
    A.withhold_inst = -1;
    A.withhold_stage = -1;
    e = cudaMemsetAsync(r->d_ctr, 0, sizeof(int) * (2 + r->n_counters), r->stream);
    if (e != cudaSuccess) return bfail(MPRK_ECUDA, std::string("batch runner: ") + cudaGetErrorString(e));
    const size_t smem = stage_smem_bytes(r->precision);
    const int grid = std::min(r->grid, r->n_items);
    batch_launch(r->precision, r->rows, grid, smem, r->stream, A);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return bfail(MPRK_ECUDA, std::string("batch runner launch: ") + cudaGetErrorString(e));
  for (int j = 0; j < count; j++) instance_count_steps(insts[j], 1);
  if (cell_stages) *cell_stages = r->cell_stages;
  return MPRK_OK;
}

bool tuned_tile_shape(long long cells, TileShape* out) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  if (g_shape.empty()) return false;
  auto it = g_shape.find(cells_bucket((double)cells));
  if (it == g_shape.end()) return false;
  *out = it->second.shape;
  return true;
}

int batch_step_on(mprk_instance* const* insts, int count, int n, cudaStream_t stream, long long* cell_stages) {
  return step_batch(insts, count, n, 2000000000LL, -1, -1, stream, cell_stages);
}

// Drop cached plans that mention an instance about to be destroyed.
void batch_forget(const void* inst) {
  std::lock_guard<std::mutex> lk(g_batch_mu);
  for (size_t j = 0; j < g_plans.size();) {
    Plan* p = g_plans[j];
    if (std::find(p->key.begin(), p->key.end(), inst) != p->key.end()) {
      if (p->stream) cudaStreamSynchronize(p->stream);
      free_plan(p);
      g_plans.erase(g_plans.begin() + j);
    } else {
      j++;
    }
  }
}
}  // namespace mprk

extern "C" {

int mprk_step_batch(mprk_instance* const* insts, int count, int n_slow_steps) {
  // about one second at 2 GHz per wait
  return step_batch(insts, count, n_slow_steps, 2000000000LL, -1, -1, nullptr, nullptr);
}

int mprk_batch_tune(mprk_instance* const* insts, int count, int reps, double out[4]) {
  if (!insts || count <= 0 || reps < 1 || !out) return bfail(MPRK_EINVAL, "bad tuning arguments");
  if (int rc = check_members(insts, count)) return rc;
  // the runs advance the states: keep them (and the step counts) to restore
  std::vector<std::vector<double>> saved(count);
  std::vector<long long> steps(count);
  for (int j = 0; j < count; j++) {
    if (!insts[j]) return bfail(MPRK_EINVAL, "NULL instance in batch");
    Geom g;
    Bufs b;
    int prec;
    cudaStream_t st;
    unsigned* sw;
    int rc = instance_view(insts[j], &g, &b, &prec, &st, &sw);
    if (rc) return rc;
    saved[j].resize((size_t)4 * g.nz * g.ny * g.nx);
    if ((rc = mprk_get_state(insts[j], saved[j].data(), MPRK_HOST))) return rc;
    steps[j] = instance_steps(insts[j]);
  }
  std::lock_guard<std::mutex> lk(g_batch_mu);
  int best_g = 0, best_c = 0, best_r = TZ, prec = 0, bucket = 0;
  double best_ms = 1e300;
  int rc = MPRK_OK;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = bfail(MPRK_ECUDA, "event create");
  // FP64 tile shapes of the 256-thread CTA: TZ rows with one thread per
  // cell, TZ / 2 rows with two; the FP32-flux tile has one shape
  int prec0 = 0;
  {
    Geom g;
    Bufs b;
    cudaStream_t st;
    unsigned* sw;
    if ((rc = instance_view(insts[0], &g, &b, &prec0, &st, &sw))) prec0 = 0;
  }
  const std::vector<int> row_choices = prec0 == 0 ? std::vector<int>{TZ, TZ / 2} : std::vector<int>{MTZ};
  // FP32 flux also times the per-stage form (tiles per item 0) with 1, 2 or
  // 4 instance groups (held in the CTAs per SM field)
  const std::vector<int> groups = prec0 == 0 ? std::vector<int>{1, 2, 4, 8, 16} : std::vector<int>{0, 1, 2, 4, 8, 16};
  for (int R : row_choices) {
    for (int G : groups) {
      for (int c = 1; c <= (G == 0 ? 4 : 3) && rc == MPRK_OK; c += (G == 0 && c == 2) ? 2 : 1) {
        Plan* p = nullptr;
        rc = build_plan(insts, count, 2000000000LL, -1, -1, nullptr, G, c, R, &p);
        if (rc) break;
        prec = p->precision;
        bucket = p->bucket;
        if (p->form == 0 && p->per_sm < c) {  // more CTAs than fit
          free_plan(p);
          continue;
        }
        cudaGraphLaunch(p->exec, p->stream);  // warm-up
        cudaEventRecord(e0, p->stream);
        for (int k = 0; k < reps; k++) cudaGraphLaunch(p->exec, p->stream);
        cudaEventRecord(e1, p->stream);
        float ms = 0.f;
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
          rc = bfail(MPRK_ECUDA, "tuning run failed");
        free_plan(p);
        if (rc == MPRK_OK && ms / reps < best_ms) {
          best_ms = ms / reps;
          best_g = G;
          best_c = c;
          best_r = R;
        }
      }
      if (rc) break;
    }
    if (rc) break;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  for (int j = 0; j < count; j++) {
    const int r2 = mprk_set_state(insts[j], saved[j].data(), MPRK_HOST);
    if (!rc) rc = r2;
    instance_count_steps(insts[j], (int)(steps[j] - instance_steps(insts[j])));
  }
  if (rc) return rc;
  {
    std::lock_guard<std::mutex> tl(g_tune_mu);
    g_tune[{prec, bucket}] = TuneVal{best_g, best_c, best_ms, best_r};
    g_tune_gpu = device_name();
  }
  out[0] = best_g;
  out[1] = best_c;
  out[2] = best_ms;
  out[3] = best_r;
  return MPRK_OK;
}

int mprk_tune_lookup(int precision, double mean_cells, int* group, int* ctas_per_sm, int* tile_rows) {
  if (!group || !ctas_per_sm || !tile_rows || precision < 0 || precision > 1 || !(mean_cells >= 1.0))
    return bfail(MPRK_EINVAL, "bad tuning lookup");
  const int bucket = cells_bucket(mean_cells);
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tune.find({precision, bucket});
  if (it == g_tune.end()) {
    *group = precision == 0 ? batch_group(precision) : 0;
    *ctas_per_sm = 0;
    *tile_rows = precision == 0 ? TZ : MTZ;
    return 0;
  }
  *group = it->second.group;
  *ctas_per_sm = it->second.per_sm;
  *tile_rows = precision == 0 ? it->second.rows : MTZ;
  return 1;
}

int mprk_tile_lookup(double cells, int* tile_rows, int* threads_per_cell) {
  if (!tile_rows || !threads_per_cell || !(cells >= 1.0)) return bfail(MPRK_EINVAL, "bad tile lookup");
  TileShape t;
  if (!tuned_tile_shape((long long)cells, &t)) return 0;
  *tile_rows = t.rows;
  *threads_per_cell = t.tpc;
  return 1;
}

int mprk_tile_tune(mprk_instance* const* insts, int count, int reps, int* entries) {
  if (!insts || count <= 0 || reps < 1 || !entries) return bfail(MPRK_EINVAL, "bad tile tuning arguments");
  // Per size bucket of a launch's cells: the summed time of each shape over
  // the instances' launches of that bucket. The launches timed are the first
  // stage (every row) and the first stage of the second fast substep (the B
  // and F rows): both read the state and write only the stage scratch, so
  // the instances' states are untouched.
  const TileShape shapes[6] = {{TZ, 1}, {TZ, 2}, {TZ / 2, 1}, {TZ / 2, 2}, {TZ / 4, 1}, {TZ / 4, 2}};
  std::map<int, std::vector<double>> tsum;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = MPRK_OK;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    rc = bfail(MPRK_ECUDA, "event create");
  for (int j = 0; j < count && rc == MPRK_OK; j++) {
    Geom g;
    Bufs b;
    int prec;
    cudaStream_t st;
    unsigned* sw;
    if (!insts[j]) { rc = bfail(MPRK_EINVAL, "NULL instance"); break; }
    if ((rc = instance_view(insts[j], &g, &b, &prec, &st, &sw))) break;
    if (prec != MPRK_FP64 || g.ny > 1) { rc = bfail(MPRK_EINVAL, "tile tuning takes 2-D FP64 instances"); break; }
    std::vector<int> stages{0};
    if (g.m > 1) stages.push_back(g.s);
    for (int stg : stages) {
      StageArgs a = stage_args(g, b, stg);
      a.status = sw;
      const int bucket = cells_bucket((double)(g.nz - a.row0) * g.nx);
      std::vector<double>& acc = tsum[bucket];
      acc.resize(6, 0.0);
      for (int k = 0; k < 6 && rc == MPRK_OK; k++) {
        cudaError_t e = launch_stage(a, 0, stage_tiles(a), st, nullptr, &shapes[k]);  // warm-up
        if (e == cudaSuccess) e = cudaEventRecord(e0, st);
        for (int r = 0; r < reps && e == cudaSuccess; r++) e = launch_stage(a, 0, stage_tiles(a), st, nullptr, &shapes[k]);
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) rc = bfail(MPRK_ECUDA, std::string("tile tuning: ") + cudaGetErrorString(e));
        acc[k] += ms / reps;
      }
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (rc) return rc;
  std::lock_guard<std::mutex> tl(g_tune_mu);
  for (const auto& kv : tsum) {
    int best = 0;
    for (int k = 1; k < 6; k++)
      if (kv.second[k] < kv.second[best]) best = k;
    g_shape[kv.first] = ShapeVal{shapes[best], kv.second[best]};
  }
  g_tune_gpu = device_name();
  *entries = (int)tsum.size();
  return MPRK_OK;
}

int mprk_tune_clear(void) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune.clear();
  g_shape.clear();
  g_tune_gpu.clear();
  return MPRK_OK;
}

int mprk_tune_save(const char* path) {
  if (!path) return bfail(MPRK_EINVAL, "NULL path");
  std::lock_guard<std::mutex> lk(g_tune_mu);
  std::string gpu;
  for (char ch : g_tune_gpu) {
    if (ch == '"' || ch == '\\') gpu += '\\';
    gpu += ch;
  }
  std::ofstream f(path);
  if (!f) return bfail(MPRK_EINVAL, std::string("cannot write ") + path);
  f << "{\"gpu\": \"" << gpu << "\", \"entries\": [";
  bool first = true;
  char buf[256];
  for (const auto& kv : g_tune) {
    snprintf(buf, sizeof buf,
             "%s\n  {\"precision\": %d, \"bucket\": %d, \"group\": %d, \"ctas_per_sm\": %d, \"tile_rows\": %d, "
             "\"ms\": %.6g}",
             first ? "" : ",", kv.first.first, kv.first.second, kv.second.group, kv.second.per_sm,
             kv.first.first == 0 ? kv.second.rows : MTZ, kv.second.ms);
    f << buf;
    first = false;
  }
  for (const auto& kv : g_shape) {
    snprintf(buf, sizeof buf,
             "%s\n  {\"stage_launch\": 1, \"bucket\": %d, \"tile_rows\": %d, \"threads_per_cell\": %d, \"ms\": %.6g}",
             first ? "" : ",", kv.first, kv.second.shape.rows, kv.second.shape.tpc, kv.second.ms);
    f << buf;
    first = false;
  }
  f << "\n]}\n";
  return f.good() ? MPRK_OK : bfail(MPRK_EINVAL, std::string("write failed: ") + path);
}

int mprk_tune_load(const char* path) {
  if (!path) return bfail(MPRK_EINVAL, "NULL path");
  std::ifstream f(path);
  if (!f) return bfail(MPRK_EINVAL, std::string("cannot read ") + path);
  std::stringstream ss;
  ss << f.rdbuf();
  const std::string t = ss.str();
  // the GPU name: the string after "gpu":
  size_t k = t.find("\"gpu\"");
  if (k == std::string::npos || (k = t.find('"', t.find(':', k) + 1)) == std::string::npos)
    return bfail(MPRK_EINVAL, "tuning file: no gpu name");
  std::string gpu;
  for (size_t j = k + 1; j < t.size() && t[j] != '"'; j++) {
    if (t[j] == '\\' && j + 1 < t.size()) j++;
    gpu += t[j];
  }
  const std::string here = device_name();
  if (!here.empty() && gpu != here)
    return bfail(MPRK_EINVAL, "tuning file measured on " + gpu + ", this device is " + here);
  auto num = [&](const std::string& obj, const char* key, double* v) {
    const size_t a = obj.find(std::string("\"") + key + "\"");
    if (a == std::string::npos) return false;
    const size_t c = obj.find(':', a);
    if (c == std::string::npos) return false;
    char* end = nullptr;
    *v = strtod(obj.c_str() + c + 1, &end);
    return end != obj.c_str() + c + 1;
  };
  std::map<std::pair<int, int>, TuneVal> table;
  std::map<int, ShapeVal> shapes;
  size_t pos = t.find("\"entries\"");
  if (pos == std::string::npos) return bfail(MPRK_EINVAL, "tuning file: no entries");
  for (;;) {
    const size_t a = t.find('{', pos), b = a == std::string::npos ? a : t.find('}', a);
    if (a == std::string::npos || b == std::string::npos) break;
    const std::string obj = t.substr(a, b - a + 1);
    double pr, bu, gr, ct, rows = TZ, tpc, sl = 0.0, ms = 0.0;
    num(obj, "ms", &ms);
    if (num(obj, "stage_launch", &sl) && sl != 0.0) {
      // a tile shape of single-instance FP64 stage launches
      if (!num(obj, "bucket", &bu) || !num(obj, "tile_rows", &rows) || !num(obj, "threads_per_cell", &tpc))
        return bfail(MPRK_EINVAL, "tuning file: incomplete tile-shape entry");
      const TileShape ts{(int)rows, (int)tpc};
      if (bu < 0 || bu > 40 || !tile_shape_valid(ts) || rows != (int)rows || tpc != (int)tpc)
        return bfail(MPRK_EINVAL, "tuning file: tile shape out of range");
      shapes[(int)bu] = ShapeVal{ts, ms};
      pos = b + 1;
      continue;
    }
    if (!num(obj, "precision", &pr) || !num(obj, "bucket", &bu) || !num(obj, "group", &gr) ||
        !num(obj, "ctas_per_sm", &ct))
      return bfail(MPRK_EINVAL, "tuning file: incomplete entry");
    num(obj, "tile_rows", &rows);
    if ((pr != 0 && pr != 1) || bu < 0 || bu > 40 || gr < (pr == 0 ? 1 : 0) || gr > 64 || ct < 0 || ct > 8 ||
        (pr == 0 && rows != TZ && rows != TZ / 2))
      return bfail(MPRK_EINVAL, "tuning file: value out of range");
    table[{(int)pr, (int)bu}] = TuneVal{(int)gr, (int)ct, ms, pr == 0 ? (int)rows : MTZ};
    pos = b + 1;
  }
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune.swap(table);
  g_shape.swap(shapes);
  g_tune_gpu = gpu;
  return MPRK_OK;
}

int mprk_batch_test_withhold(mprk_instance* const* insts, int count, int inst_index, int stage,
                             long long wait_cycles) {
  if (inst_index < 0 || inst_index >= count || stage < 0) return bfail(MPRK_EINVAL, "bad withhold target");
  return step_batch(insts, count, 1, wait_cycles, inst_index, stage, nullptr, nullptr);
}

}  // extern "C"
