// capi.cu -- the C ABI of include/rasp.h: batch state store, loading of
// programs and tapes (c_0 of Sec. 2.1), scheduling by memory-size bucket,
// read-back and checkpoint restore.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "../../include/rasp.h"
#include "engine.cuh"
#include "internal.h"

using namespace rasp;

bool rasp::inject_alloc_failure() {
  const char* v = getenv("RASP_FAULT_INJECT");
  return v && strcmp(v, "alloc") == 0;
}

bool rasp::inject_wait_expiry() {
  const char* v = getenv("RASP_FAULT_INJECT");
  return v && strcmp(v, "wait") == 0;
}

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

#define CK(call)                                                                         \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess) return fail(RASP_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

constexpr size_t ALIGN = 256;
inline size_t align_up(size_t x) { return (x + ALIGN - 1) & ~(ALIGN - 1); }

// Memory-size buckets: VMs whose n falls in the same class share a slot size.
constexpr uint32_t kBucketBounds[] = {64, 128, 256, 512, 768, 1024, 2048, 4096, 1u << 31};
constexpr int kNumBuckets = sizeof(kBucketBounds) / sizeof(kBucketBounds[0]);

struct Bucket {
  uint32_t first = 0;      // position in the id list
  uint32_t count = 0;
  uint32_t ncap = 0;       // largest padded n in the bucket
  uint32_t sched = 0;      // RASP_SCHED_PLAIN / PERSIST / PERSIST_GL
  PersistShape shape{};
};

// One launch: adjacent buckets on the HBM-slab persistent schedule share one
// queue (that schedule does not depend on n); others launch per bucket.
struct Group {
  uint32_t first = 0;
  uint32_t count = 0;
  uint32_t sched = 0;
  PersistShape shape{};
};

// A schedule and launch shape chosen for one bucket by the autotuner (in
// place of the batch-wide rasp_config settings).
struct BucketPlan {
  bool set = false;
  uint32_t sched = 0, epoch = 0, warps = 0, ctas = 0;
  bool block = false;      // the per-step form instead of the epoch loop
};

struct Layout {
  size_t off_i, off_a, off_steps, off_cap, off_status, off_uhead, off_ylen, off_n, off_memoff;
  size_t off_mem, off_prog, off_progoff, off_progvm, off_tape, off_y, off_ids, off_heads, off_err,
      off_hist, off_stats, off_dirty, off_pvoff, off_pvids, off_thist, off_ids2, off_rcount, off_topk;
  size_t total;
};

}  // namespace

struct rasp_batch {
  rasp_config cfg{};
  cudaStream_t stream = nullptr;
  uint32_t V = 0;
  uint32_t ell = 0, s = 0, ellp = 0, sp = 0;
  uint64_t wmask = ~0ull;
  std::vector<uint32_t> h_n;
  std::vector<uint64_t> h_memoff;
  uint64_t mem_words = 0;      // sum of padded n
  Layout L{};
  char* base = nullptr;
  bool owns = false;
  DevState S{};
  uint64_t* d_prog = nullptr;
  // Programs loaded as 4-byte words are kept as such in the upper half of
  // the program area when they fit beside their widened copy: the pack
  // reads them there, and d_prog is filled (widened) only when a kernel
  // that reads 8-byte program words needs it (prog64_valid).
  const int32_t* prog32 = nullptr;
  uint64_t prog_words = 0;
  bool prog64_valid = true;
  uint64_t* d_progoff = nullptr;
  uint32_t* d_progvm = nullptr;
  uint32_t* d_ids = nullptr;
  uint32_t* d_heads = nullptr;
  int* d_err = nullptr;
  unsigned long long* d_hist = nullptr;
  unsigned long long* d_stats = nullptr;
  uint64_t* d_cap = nullptr;
  bool shared_programs = false;
  bool programs_loaded = false, inputs_loaded = false;
  std::vector<uint32_t> h_ids;       // queue order: bucket-contiguous, sorted within each launch group
  std::vector<uint32_t> h_ids_base;  // bucket-contiguous, VM id order within a bucket
  std::vector<uint64_t> h_caps;      // per-VM caps (empty: all uncapped)
  std::vector<Bucket> buckets;
  std::vector<Group> groups;
  std::vector<BucketPlan> over;      // per-bucket autotuned choices (empty: the batch-wide settings)
  uint64_t launches = 0;
  // CUDA graphs of rasp_run, one per budget (RASP_CUDA_GRAPH)
  cudaStream_t cap_stream = nullptr;
  std::vector<std::pair<uint64_t, cudaGraphExec_t>> graphs;
  std::string tuned;           // JSON report of the last rasp_autotune
  // shared programs: VMs grouped by program (CSR) and the longest program
  uint32_t* d_pvoff = nullptr;
  uint32_t* d_pvids = nullptr;
  uint32_t num_programs = 0;
  uint32_t max_plen = 0;
  bool dirty_valid = false;    // codedirty is up to date (only the shared kernel tracks it)
  bool code_lazy = false;      // slabs of VMs with codedirty = 0 lack their program words (lazy pack)
  bool tuned_block = false;    // autotuned: the SMEM-staged schedule one step at a time
  bool narrow = false;         // M in 4-byte words (w <= 32)
  bool uhead_pending = false;  // u_0 = 0 owed since rasp_load_inputs (done by the pack or before the next use)
  bool ids_uploaded = false;   // d_ids holds h_ids
  bool ids_base = true;        // h_ids is h_ids_base (bucket order, no cap-class sort)
  uint64_t max_cap = ~0ull;    // largest step cap of the batch (no VM runs further)
  uint32_t* d_ids2 = nullptr;  // compacted queue between budget rounds
  uint32_t* d_rcount = nullptr;
  bool planned = true;         // buckets have schedules and launch groups
};

namespace {

int validate_config(const rasp_config* cfg, uint64_t num_vms, const uint32_t* mem_words) {
  if (!cfg) return fail(RASP_EINVAL, "config is NULL");
  if (cfg->word_bits < 2 || cfg->word_bits > 64) return fail(RASP_EINVAL, "word_bits must be in 2..64");
  if (cfg->reserved) return fail(RASP_EINVAL, "rasp_config.reserved must be 0");
  if (cfg->semantics != RASP_WRAP && cfg->semantics != RASP_CHECKED)
    return fail(RASP_EINVAL, "unknown semantics %u", cfg->semantics);
  if (cfg->semantics == RASP_CHECKED && cfg->word_bits != 64)
    return fail(RASP_EINVAL, "CHECKED semantics needs word_bits = 64");
  if (num_vms == 0 || num_vms >= (1ull << 32)) return fail(RASP_EINVAL, "num_vms must be in 1..2^32-1");
  if (!mem_words) return fail(RASP_EINVAL, "mem_words is NULL");
  const uint32_t sched = cfg->flags & RASP_SCHED_MASK;
  if (sched != RASP_SCHED_AUTO && sched != RASP_SCHED_PLAIN && sched != RASP_SCHED_PERSIST &&
      sched != RASP_SCHED_PERSIST_GL && sched != RASP_SCHED_SHARED)
    return fail(RASP_EINVAL, "unknown schedule flag 0x%x", sched);
  if (cfg->flags & RASP_ISA_CLASSIC) {
    if (sched != RASP_SCHED_AUTO && sched != RASP_SCHED_PLAIN && sched != RASP_SCHED_PERSIST_GL)
      return fail(RASP_EINVAL, "the classic opcode set runs on the plain and HBM-slab persistent schedules only");
    if (cfg->flags & RASP_DISPATCH_VOTE)
      return fail(RASP_EINVAL, "the classic opcode set uses the select dispatch only");
  }
  if (cfg->word_bits < 64) {
    const uint64_t lim = 1ull << cfg->word_bits;
    if (cfg->in_cap >= lim || cfg->out_cap >= lim)
      return fail(RASP_EINVAL, "l and s must be representable in w bits");
  }
  for (uint64_t v = 0; v < num_vms; ++v)
    if (mem_words[v] == 0 || mem_words[v] >= (1u << 31))
      return fail(RASP_EINVAL, "mem_words[%llu] = %u is outside 1..2^31-1", (unsigned long long)v, mem_words[v]);
  return RASP_OK;
}

// Blocks of the first top-k pass (each takes at least 1024 fresh candidates per tile).
uint64_t topk_blocks(uint64_t V) { return std::min<uint64_t>(kMaxTopBlocks, (V + 1023) / 1024); }

// M in 4-byte words: w <= 32 on the schedules that read M through a narrow
// view (plain and HBM-slab persistent; the shared-program and SMEM-staged
// kernels keep 8-byte words, and so do the serving pool's batches).
bool narrow_layout(const rasp_config* cfg, bool plan) {
  const uint32_t sched = cfg->flags & RASP_SCHED_MASK;
  return plan && cfg->word_bits <= 32 && sched != RASP_SCHED_SHARED && sched != RASP_SCHED_PERSIST;
}

Layout make_layout(uint64_t V, uint64_t mem_words, uint32_t ellp, uint32_t sp, uint32_t word_bytes) {
  Layout L{};
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t r = o;
    o = align_up(o + bytes);
    return r;
  };
  L.off_i = take(8 * V);
  L.off_a = take(8 * V);
  L.off_steps = take(8 * V);
  L.off_cap = take(8 * V);
  L.off_status = take(V);
  L.off_uhead = take(4 * V);
  L.off_ylen = take(4 * V);
  L.off_n = take(4 * V);
  L.off_memoff = take(8 * V);
  L.off_mem = take((uint64_t)word_bytes * mem_words);
  L.off_prog = take(8 * mem_words);           // programs never exceed the M arena
  L.off_progoff = take(8 * (V + 1));
  L.off_progvm = take(4 * V);
  L.off_tape = take(8 * V * (uint64_t)ellp);
  L.off_y = take(8 * V * (uint64_t)sp);
  L.off_ids = take(4 * V);
  L.off_heads = take(8 * kNumBuckets);
  L.off_err = take(16);
  L.off_hist = take(8 * 10);
  L.off_stats = take(8 * 6);
  L.off_dirty = take(V);
  L.off_pvoff = take(4 * (V + 1));
  L.off_pvids = take(4 * V);
  L.off_thist = take(8 * (2 * kMaxHistBins + 1 + 4));   // edges, counts, other
  L.off_ids2 = take(4 * V);                             // compacted queue between budget rounds
  L.off_rcount = take(4 * kNumBuckets);                 // its length, per launch group
  L.off_topk = take(sizeof(TopCand) * (topk_blocks(V) + 1) * kMaxTopK);  // top-k candidates, result
  L.total = o;
  return L;
}

uint32_t even(uint32_t x) { return (x + 1u) & ~1u; }

StepVariant variant_of(const rasp_batch* b) {
  StepVariant v{};
  v.masked = b->cfg.word_bits < 64;
  v.checked = b->cfg.semantics == RASP_CHECKED;
  v.hist = (b->cfg.flags & RASP_COLLECT_STATS) != 0;
  v.vote = (b->cfg.flags & RASP_DISPATCH_VOTE) != 0;
  v.classic = (b->cfg.flags & RASP_ISA_CLASSIC) != 0;
  v.block = (b->cfg.flags & RASP_STEP_BLOCK) != 0;
  v.narrow = b->narrow;
  return v;
}

// Choose a schedule and launch shape per bucket: the batch-wide settings of
// rasp_config, or the bucket's own autotuned choice.
void plan_buckets(rasp_batch* b) {
  const StepVariant var = variant_of(b);
  for (size_t bi = 0; bi < b->buckets.size(); ++bi) {
    Bucket& k = b->buckets[bi];
    if (!k.count) continue;
    const bool own = bi < b->over.size() && b->over[bi].set;
    const uint32_t cfg_epoch = own ? b->over[bi].epoch : b->cfg.epoch;
    const uint32_t cfg_warps = own ? b->over[bi].warps : b->cfg.warps_per_cta;
    const uint32_t cfg_ctas = own ? b->over[bi].ctas : b->cfg.ctas_per_sm;
    uint32_t sched = own ? b->over[bi].sched : (b->cfg.flags & RASP_SCHED_MASK);
    if (sched == RASP_SCHED_SHARED) {
      k.sched = sched;                     // one launch over programs, see build_groups
      continue;
    }
    const uint32_t slot = [&] {
      uint32_t w = k.ncap + b->ellp + b->sp;
      w = even(w);
      if ((w & 3u) == 0) w += 2u;          // stride = 2 mod 4 words: conflict-free 16-byte rows
      return w;
    }();
    const size_t staged_bytes = (32ull + 32ull * slot) * 8ull;   // 64-bit: slot reaches 2^31
    // default before autotuning: persistent workers over HBM-resident slabs
    // (measured fastest on the 256-word template workload)
    if (sched == RASP_SCHED_AUTO) sched = RASP_SCHED_PERSIST_GL;
    if (sched == RASP_SCHED_PERSIST && (staged_bytes > 220u * 1024u || b->narrow)) sched = RASP_SCHED_PERSIST_GL;
    k.sched = sched;
    PersistShape& sh = k.shape;
    sh = PersistShape{};
    sh.ncap = k.ncap;
    sh.slot_words = slot;
    sh.epoch = cfg_epoch ? cfg_epoch : 32u;
    // the one-step form of an autotuned staged plan; a bucket too large for
    // shared memory keeps the HBM-slab loop
    sh.block = (own ? b->over[bi].block : b->tuned_block) && sched == RASP_SCHED_PERSIST;
    if (sched == RASP_SCHED_PERSIST) {
      sh.staged = true;
      sh.warps = 1;
      sh.refill_min = 8;
    } else {
      sh.staged = false;
      sh.warps = 4;
      sh.refill_min = 1;
      sh.epoch = cfg_epoch ? cfg_epoch : 128u;
      sh.idle_exit = std::min<uint32_t>(b->cfg.refill_min, 32u);   // epoch loop: end an epoch after this many stops
    }
    if (cfg_warps) sh.warps = std::min<uint32_t>(cfg_warps, 8u);
    if (!sh.staged) sh.warps = std::min<uint32_t>(sh.warps, 4u);   // k_persist_gl: at most 128 threads
    if (b->cfg.refill_min) sh.refill_min = std::min<uint32_t>(b->cfg.refill_min, 32u);
    if (sched == RASP_SCHED_PLAIN) plain_configure(var);
    if (sched != RASP_SCHED_PLAIN) {
      if (persist_configure(var, sh) == 0) {
        plain_configure(var);
        k.sched = RASP_SCHED_PLAIN;        // cannot be resident: fall back to the plain form
      } else if (cfg_ctas && cfg_ctas < sh.ctas_per_sm) {
        sh.grid = sh.grid / sh.ctas_per_sm * cfg_ctas;
        sh.ctas_per_sm = cfg_ctas;
      }
    }
  }
}

// Power-of-two class of a step cap (0 for caps 0 and 1, 64 for no cap).
inline uint32_t cap_class(uint64_t c) { return c ? 64u - (uint32_t)__builtin_clzll(c) : 0u; }

// Queue order for the current launch groups: every group's range holds
// exactly the VMs of its buckets; inside a group, VMs with the larger cap
// class come first (the largest work starts first), in VM id order within a
// class -- a stable counting sort, linear in the batch. Uploads the order
// only when it changed.
int order_ids(rasp_batch* b) {
  if (b->h_caps.empty() && b->ids_base && b->ids_uploaded) return RASP_OK;   // uniform caps: bucket order
  std::vector<uint32_t> ids = b->h_ids_base;
  if (!b->h_caps.empty()) {
    const std::vector<uint64_t>& caps = b->h_caps;
    std::vector<uint32_t> tmp;
    std::vector<Group> whole;
    if (b->groups.empty()) {                   // not planned: one range, the whole queue
      whole.resize(1);
      whole[0].count = b->V;
    }
    for (const Group& k : b->groups.empty() ? whole : b->groups) {
      if (k.count < 2) continue;
      uint32_t cnt[66] = {0};
      for (uint32_t q = k.first; q < k.first + k.count; ++q) cnt[64u - cap_class(caps[ids[q]]) + 1u]++;
      for (int c = 1; c < 66; ++c) cnt[c] += cnt[c - 1];
      tmp.assign(ids.begin() + k.first, ids.begin() + k.first + k.count);
      for (uint32_t v : tmp) ids[k.first + cnt[64u - cap_class(caps[v])]++] = v;
    }
  }
  if (ids == b->h_ids && b->ids_uploaded) return RASP_OK;
  b->h_ids.swap(ids);
  b->ids_base = b->h_caps.empty();
  CK(cudaMemcpyAsync(b->d_ids, b->h_ids.data(), 4ull * b->V, cudaMemcpyHostToDevice, b->stream));
  CK(cudaStreamSynchronize(b->stream));
  b->ids_uploaded = true;
  return RASP_OK;
}

void build_groups(rasp_batch* b) {
  b->groups.clear();
  if ((b->cfg.flags & RASP_SCHED_MASK) == RASP_SCHED_SHARED) {
    Group g;
    g.first = 0;
    g.count = b->V;
    g.sched = RASP_SCHED_SHARED;
    b->groups.push_back(g);
    return;
  }
  for (const Bucket& k : b->buckets) {
    if (!k.count) continue;
    const PersistShape& gs = b->groups.empty() ? k.shape : b->groups.back().shape;
    const bool same_shape = gs.warps == k.shape.warps && gs.epoch == k.shape.epoch && gs.grid == k.shape.grid &&
                            gs.ctas_per_sm == k.shape.ctas_per_sm && gs.idle_exit == k.shape.idle_exit &&
                            gs.block == k.shape.block;
    if (!b->groups.empty() && k.sched == RASP_SCHED_PERSIST_GL && b->groups.back().sched == RASP_SCHED_PERSIST_GL &&
        same_shape && b->groups.back().first + b->groups.back().count == k.first) {
      b->groups.back().count += k.count;
      continue;
    }
    Group g;
    g.first = k.first;
    g.count = k.count;
    g.sched = k.sched;
    g.shape = k.shape;
    b->groups.push_back(g);
  }
}

// The shared-program schedule reads program words from the program itself
// until a VM writes one of them, so its c_0 writes only the data words.
bool pack_lazy(const rasp_batch* b) {
  return b->planned && (b->cfg.flags & RASP_SCHED_MASK) == RASP_SCHED_SHARED;
}

// The 8-byte program words of programs kept as 4-byte words, before a
// kernel other than the pack reads them (materialize, the shared-program
// schedule).
cudaError_t ensure_prog64(rasp_batch* b, cudaStream_t st) {
  if (b->prog64_valid) return cudaSuccess;
  b->prog64_valid = true;
  return launch_widen(b->prog32, b->d_prog, b->prog_words, st);
}

// Before anything but the shared-program kernel reads the slabs of a lazily
// packed batch: the program words of every VM whose slab lacks them.
cudaError_t materialize(rasp_batch* b, cudaStream_t st) {
  if (!b->code_lazy) return cudaSuccess;
  const cudaError_t e = ensure_prog64(b, st);
  if (e != cudaSuccess) return e;
  b->code_lazy = false;
  return launch_materialize(b->S, b->d_prog, b->d_progoff, b->shared_programs ? b->d_progvm : nullptr, b->V,
                            b->wmask, st);
}

// rasp_load_inputs resets u_0 without queuing a kernel (so that the next
// load's wait for its host copies cannot stall behind kernels of other
// batches): the pack does it, or this before u_0 is next read.
cudaError_t apply_uhead_reset(rasp_batch* b, cudaStream_t st) {
  if (!b->uhead_pending) return cudaSuccess;
  b->uhead_pending = false;
  return fill_bytes(b->S.uhead, 0, 4ull * b->V, st);
}

int replan(rasp_batch* b);

int check_device_error(rasp_batch* b) {
  int err = 0;
  CK(cudaMemcpyAsync(&err, b->d_err, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
  CK(cudaStreamSynchronize(b->stream));
  if (err) return fail(RASP_EDEVICE, "a kernel reported internal error %d (%s)", err,
                       err == ERR_SLOT ? "VM larger than its bucket's slot"
                                       : (err == ERR_RING ? "ring entry outside the slot table" : "bounded wait expired"));
  return RASP_OK;
}

}  // namespace

const DevState& rasp::batch_dev_state(const rasp_batch* b) { return b->S; }

Params rasp::batch_params(const rasp_batch* b) {
  Params P{};
  P.wmask = b->wmask;
  P.budget = ~0ull;
  P.ell = b->ell;
  P.s = b->s;
  P.ellp = b->ellp;
  P.sp = b->sp;
  P.err = b->d_err;
  P.hist = b->d_hist;
  return P;
}

const uint32_t* rasp::batch_queue(const rasp_batch* b) { return b->d_ids; }

extern "C" {

const char* rasp_last_error(void) { return g_err.c_str(); }

const char* rasp_version(void) { return "rasp_gb300 1.0 (sm_103a)"; }

int rasp_batch_bytes(const rasp_config* cfg, uint64_t num_vms, const uint32_t* mem_words, uint64_t* out_bytes) {
  int rc = validate_config(cfg, num_vms, mem_words);
  if (rc) return rc;
  if (!out_bytes) return fail(RASP_EINVAL, "out_bytes is NULL");
  uint64_t mw = 0;
  for (uint64_t v = 0; v < num_vms; ++v) mw += even(mem_words[v]);
  *out_bytes = make_layout(num_vms, mw, even(cfg->in_cap), even(cfg->out_cap), narrow_layout(cfg, true) ? 4u : 8u).total +
               ALIGN;
  return RASP_OK;
}

int rasp_batch_create(const rasp_config* cfg, uint64_t num_vms, const uint32_t* mem_words, rasp_batch** out) {
  return rasp::create_batch(cfg, num_vms, mem_words, true, out);
}

}  // extern "C"

// With plan = false the launch plan (schedules per bucket) is made by the
// first rasp_run instead (the serving pool's batches are never run by
// rasp_run: its kernel schedules their VMs).
int rasp::create_batch(const rasp_config* cfg, uint64_t num_vms, const uint32_t* mem_words, bool plan,
                       rasp_batch** out) {
  if (!out) return fail(RASP_EINVAL, "out is NULL");
  *out = nullptr;
  int rc = validate_config(cfg, num_vms, mem_words);
  if (rc) return rc;
  rasp_batch* b = new (std::nothrow) rasp_batch();
  if (!b) return fail(RASP_ENOMEM, "host allocation failed");
  b->cfg = *cfg;
  b->stream = (cudaStream_t)cfg->stream;
  b->V = (uint32_t)num_vms;
  b->ell = cfg->in_cap;
  b->s = cfg->out_cap;
  b->ellp = even(cfg->in_cap);
  b->sp = even(cfg->out_cap);
  b->wmask = cfg->word_bits >= 64 ? ~0ull : ((1ull << cfg->word_bits) - 1ull);
  b->h_n.assign(mem_words, mem_words + num_vms);
  b->h_memoff.resize(num_vms);
  uint64_t off = 0;
  for (uint64_t v = 0; v < num_vms; ++v) {
    b->h_memoff[v] = off;
    off += even(mem_words[v]);
  }
  b->mem_words = off;
  b->narrow = narrow_layout(cfg, plan);
  b->L = make_layout(num_vms, off, b->ellp, b->sp, b->narrow ? 4u : 8u);
  if (cfg->arena) {
    const uintptr_t p = (uintptr_t)cfg->arena;
    const uintptr_t aligned = (p + ALIGN - 1) & ~(uintptr_t)(ALIGN - 1);
    if (aligned - p + b->L.total > cfg->arena_bytes) {
      delete b;
      return fail(RASP_ENOMEM, "arena of %llu bytes is smaller than the %llu the batch needs",
                  (unsigned long long)cfg->arena_bytes, (unsigned long long)(b->L.total + ALIGN));
    }
    b->base = (char*)aligned;
    b->owns = false;
  } else {
    void* p = nullptr;
    if (inject_alloc_failure()) {
      delete b;
      return fail(RASP_ENOMEM, "injected allocation failure (RASP_FAULT_INJECT=alloc)");
    }
    cudaError_t e = cudaMalloc(&p, b->L.total);
    if (e != cudaSuccess) {
      cudaGetLastError();
      delete b;
      return fail(RASP_ENOMEM, "cudaMalloc(%llu) failed: %s", (unsigned long long)b->L.total, cudaGetErrorString(e));
    }
    b->base = (char*)p;
    b->owns = true;
  }
  const Layout& L = b->L;
  char* B = b->base;
  DevState& S = b->S;
  S.i = (uint64_t*)(B + L.off_i);
  S.a = (uint64_t*)(B + L.off_a);
  S.steps = (uint64_t*)(B + L.off_steps);
  b->d_cap = (uint64_t*)(B + L.off_cap);
  S.cap = b->d_cap;
  S.status = (uint8_t*)(B + L.off_status);
  S.uhead = (uint32_t*)(B + L.off_uhead);
  S.ylen = (uint32_t*)(B + L.off_ylen);
  S.n = (const uint32_t*)(B + L.off_n);
  S.mem_off = (const uint64_t*)(B + L.off_memoff);
  S.mem = (uint64_t*)(B + L.off_mem);
  S.mem32 = b->narrow ? (uint32_t*)(B + L.off_mem) : nullptr;
  S.tape = (const uint64_t*)(B + L.off_tape);
  S.y = (uint64_t*)(B + L.off_y);
  b->d_prog = (uint64_t*)(B + L.off_prog);
  b->d_progoff = (uint64_t*)(B + L.off_progoff);
  b->d_progvm = (uint32_t*)(B + L.off_progvm);
  b->d_ids = (uint32_t*)(B + L.off_ids);
  b->d_heads = (uint32_t*)(B + L.off_heads);
  b->d_err = (int*)(B + L.off_err);
  b->d_hist = (unsigned long long*)(B + L.off_hist);
  b->d_stats = (unsigned long long*)(B + L.off_stats);
  S.codedirty = (uint8_t*)(B + L.off_dirty);
  b->d_pvoff = (uint32_t*)(B + L.off_pvoff);
  b->d_pvids = (uint32_t*)(B + L.off_pvids);
  b->d_ids2 = (uint32_t*)(B + L.off_ids2);
  b->d_rcount = (uint32_t*)(B + L.off_rcount);

  // buckets by memory size (stable: VM id order within a bucket)
  std::vector<uint32_t> cls(num_vms);
  std::vector<uint32_t> counts(kNumBuckets, 0), ncap(kNumBuckets, 0);
  for (uint64_t v = 0; v < num_vms; ++v) {
    int k = 0;
    while (even(mem_words[v]) > kBucketBounds[k]) ++k;
    cls[v] = (uint32_t)k;
    counts[k]++;
    ncap[k] = std::max(ncap[k], even(mem_words[v]));
  }
  b->buckets.resize(kNumBuckets);
  uint32_t pos = 0;
  for (int k = 0; k < kNumBuckets; ++k) {
    b->buckets[k].first = pos;
    b->buckets[k].count = counts[k];
    b->buckets[k].ncap = ncap[k];
    pos += counts[k];
  }
  b->h_ids.resize(num_vms);
  std::vector<uint32_t> fill(kNumBuckets, 0);
  for (uint64_t v = 0; v < num_vms; ++v) {
    const uint32_t k = cls[v];
    b->h_ids[b->buckets[k].first + fill[k]++] = (uint32_t)v;
  }
  b->h_ids_base = b->h_ids;
  if (plan) {
    plan_buckets(b);
    build_groups(b);
  }
  b->planned = plan;
  if (cfg->flags & RASP_CUDA_GRAPH) {
    if (cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      if (b->owns) cudaFree(b->base);
      delete b;
      return fail(RASP_ECUDA, "cannot create the capture stream");
    }
  }

  cudaStream_t st = b->stream;
  auto cleanup_fail = [&](int code) {
    if (b->owns) cudaFree(b->base);
    delete b;
    return code;
  };
#define CKC(call)                                                                              \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess) return cleanup_fail(fail(RASP_ECUDA, "%s: %s", #call, cudaGetErrorString(e_))); \
  } while (0)
  CKC(cudaMemcpyAsync((void*)S.n, mem_words, 4 * num_vms, cudaMemcpyHostToDevice, st));
  CKC(cudaMemcpyAsync((void*)S.mem_off, b->h_memoff.data(), 8 * num_vms, cudaMemcpyHostToDevice, st));
  CKC(cudaMemcpyAsync(b->d_ids, b->h_ids.data(), 4 * num_vms, cudaMemcpyHostToDevice, st));
  b->ids_uploaded = true;
  CKC(fill_bytes(b->base + L.off_status, RASP_RUNNING, num_vms, st));
  CKC(fill_bytes(b->d_err, 0, 16, st));
  CKC(fill_bytes(b->d_hist, 0, 8 * 10, st));
  CKC(fill_bytes(b->d_cap, 0xff, 8 * num_vms, st));
  CKC(cudaStreamSynchronize(st));
#undef CKC
  *out = b;
  g_err.clear();
  return RASP_OK;
}

extern "C" {

int rasp_load_programs(rasp_batch* b, const int64_t* words, const uint64_t* offsets, uint64_t num_programs,
                       const uint32_t* prog_of_vm) {
  return rasp::load_programs(b, words, 8, offsets, num_programs, prog_of_vm);
}

int rasp_load_programs_i32(rasp_batch* b, const int32_t* words, const uint64_t* offsets, uint64_t num_programs,
                           const uint32_t* prog_of_vm) {
  return rasp::load_programs(b, words, 4, offsets, num_programs, prog_of_vm);
}

}  // extern "C"

// Programs given as 8-byte words are copied into the program area; 4-byte
// words are copied into the M arena (which the pack overwrites anyway) and
// widened on the device, with sign extension, once the checks have passed.
int rasp::load_programs(rasp_batch* b, const void* words, int word_size, const uint64_t* offsets,
                        uint64_t num_programs, const uint32_t* prog_of_vm) {
  if (!b) return fail(RASP_EINVAL, "batch is NULL");
  if (!offsets || num_programs == 0) return fail(RASP_EINVAL, "offsets NULL or no programs");
  if (!prog_of_vm && num_programs != b->V)
    return fail(RASP_EINVAL, "without prog_of_vm there must be one program per VM (%llu != %u)",
                (unsigned long long)num_programs, b->V);
  if (num_programs > b->V) return fail(RASP_EINVAL, "more programs (%llu) than VMs (%u)",
                                       (unsigned long long)num_programs, b->V);
  if (offsets[0] != 0) return fail(RASP_EINVAL, "offsets[0] must be 0");
  const uint64_t total = offsets[num_programs];
  if (total > b->mem_words) return fail(RASP_EINVAL, "programs (%llu words) exceed the batch memory", (unsigned long long)total);
  if (total && !words) return fail(RASP_EINVAL, "words is NULL");
  // The copies go out first and the per-program checks run on the host while
  // they are in flight (the copies stay inside the batch's program area
  // whatever the offsets say). A failed check discards the programs: the
  // copy has already replaced the earlier ones.
  //
  // 4-byte words are kept in the upper half of the program area, at word
  // offset h = mem_words rounded up to even (8-byte aligned), when their
  // widened copy [0, 8 total) bytes stays below that offset (2 total <= h)
  // and they end inside the area: the pack then reads them there and the
  // widening waits until a kernel needs 8-byte words. Otherwise they are
  // staged in the M arena (>= 4 total bytes, overwritten by the pack) and
  // widened into the program area before the pack.
  cudaStream_t st = b->stream;
  const uint64_t h = (b->mem_words + 1ull) & ~1ull;
  const bool keep32 = word_size == 4 && 2ull * total <= h && 4ull * (h + total) <= 8ull * b->mem_words;
  int32_t* staged = keep32 ? reinterpret_cast<int32_t*>(b->d_prog) + h : reinterpret_cast<int32_t*>(b->S.mem);
  if (total)
    CK(cudaMemcpyAsync(word_size == 8 ? (void*)b->d_prog : (void*)staged, words, (size_t)word_size * total,
                       cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(b->d_progoff, offsets, 8 * (num_programs + 1), cudaMemcpyHostToDevice, st));
  if (prog_of_vm) CK(cudaMemcpyAsync(b->d_progvm, prog_of_vm, 4ull * b->V, cudaMemcpyHostToDevice, st));
  b->programs_loaded = false;
  uint32_t max_plen = 0;
  int bad = RASP_OK;
  for (uint64_t p = 0; p < num_programs && !bad; ++p) {
    const uint64_t len = offsets[p + 1] - offsets[p];
    if (offsets[p + 1] < offsets[p])
      bad = fail(RASP_EINVAL, "offsets decrease at program %llu", (unsigned long long)p);
    else if (len & 1ull)
      bad = fail(RASP_EINVAL, "program %llu has odd length (instructions are word pairs)", (unsigned long long)p);
    else if (!prog_of_vm && len > b->h_n[p])
      bad = fail(RASP_EINVAL, "program of VM %llu has %llu words > n = %u (need 2m <= n)", (unsigned long long)p,
                 (unsigned long long)len, b->h_n[p]);
    else if (len > max_plen)
      max_plen = (uint32_t)len;
  }
  for (uint32_t v = 0; prog_of_vm && v < b->V && !bad; ++v) {
    const uint64_t p = prog_of_vm[v];
    if (p >= num_programs)
      bad = fail(RASP_EINVAL, "prog_of_vm[%u] = %llu out of range", v, (unsigned long long)p);
    else if (offsets[p + 1] - offsets[p] > b->h_n[v])
      bad = fail(RASP_EINVAL, "program of VM %u has %llu words > n = %u (need 2m <= n)", v,
                 (unsigned long long)(offsets[p + 1] - offsets[p]), b->h_n[v]);
  }
  if (bad) {
    cudaStreamSynchronize(st);   // the caller's buffers are read before the call returns
    return bad;
  }
  b->shared_programs = prog_of_vm != nullptr;
  b->max_plen = max_plen;
  b->num_programs = (uint32_t)num_programs;
  if (prog_of_vm || (b->cfg.flags & RASP_SCHED_MASK) == RASP_SCHED_SHARED) {
    // VMs grouped by program (counting sort), for the shared-program schedule
    std::vector<uint32_t> pvoff(num_programs + 1, 0), pvids(b->V);
    for (uint32_t v = 0; v < b->V; ++v) pvoff[(prog_of_vm ? prog_of_vm[v] : v) + 1]++;
    for (uint64_t p = 0; p < num_programs; ++p) pvoff[p + 1] += pvoff[p];
    std::vector<uint32_t> fillp(pvoff.begin(), pvoff.end() - 1);
    for (uint32_t v = 0; v < b->V; ++v) pvids[fillp[prog_of_vm ? prog_of_vm[v] : v]++] = v;
    if (b->max_plen * 8ull > 200ull * 1024ull && (b->cfg.flags & RASP_SCHED_MASK) == RASP_SCHED_SHARED) {
      cudaStreamSynchronize(st);
      return fail(RASP_EINVAL, "shared-program schedule: a program of %u words does not fit in shared memory",
                  b->max_plen);
    }
    CK(cudaMemcpyAsync(b->d_pvoff, pvoff.data(), 4 * pvoff.size(), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(b->d_pvids, pvids.data(), 4ull * b->V, cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));
  }
  CK(cudaStreamSynchronize(st));   // the caller's buffers are read before the call returns
  // widening, like the pack, is left queued on the stream: it may have to
  // wait for SMs that another batch's run holds, and the host need not
  b->prog32 = keep32 && total ? staged : nullptr;
  b->prog_words = total;
  b->prog64_valid = !b->prog32;
  if (word_size == 4 && total && !keep32) CK(launch_widen(staged, b->d_prog, total, st));
  CK(fill_bytes(b->d_hist, 0, 8 * 10, st));
  b->code_lazy = pack_lazy(b);
  CK(launch_pack(b->S, b->d_prog, b->prog32, b->d_progoff, b->shared_programs ? b->d_progvm : nullptr, b->V,
                 b->wmask, b->sp, b->code_lazy, st));
  b->uhead_pending = false;        // the pack resets u_0
  b->programs_loaded = true;
  b->dirty_valid = true;
  g_err.clear();
  return RASP_OK;
}

extern "C" {

int rasp_load_inputs(rasp_batch* b, const int64_t* tape, const uint64_t* offsets, const uint64_t* caps) {
  if (!b) return fail(RASP_EINVAL, "batch is NULL");
  if (!offsets) return fail(RASP_EINVAL, "offsets is NULL");
  if (offsets[0] != 0) return fail(RASP_EINVAL, "offsets[0] must be 0");
  if (offsets[b->V] && !tape) return fail(RASP_EINVAL, "tape is NULL");
  cudaStream_t st = b->stream;
  uint64_t* d_tape = (uint64_t*)b->S.tape;
  const bool masked = b->wmask != ~0ull;
  // Every tape exactly l words long (l even, w = 64): one copy of the caller's
  // array, sent before the per-VM checks (which then also prove that every
  // length is l: none exceeds l and they sum to V l). A failed check discards
  // the inputs: the copy has already replaced the earlier ones.
  const bool regular = b->ellp && !masked && b->ell == b->ellp && offsets[b->V] == (uint64_t)b->V * b->ellp;
  if (regular) CK(cudaMemcpyAsync(d_tape, tape, 8ull * b->V * b->ellp, cudaMemcpyHostToDevice, st));
  if (caps) CK(cudaMemcpyAsync(b->d_cap, caps, 8ull * b->V, cudaMemcpyHostToDevice, st));
  b->inputs_loaded = false;
  int bad = RASP_OK;
  for (uint32_t v = 0; v < b->V && !bad; ++v) {
    if (offsets[v + 1] < offsets[v]) bad = fail(RASP_EINVAL, "offsets decrease at VM %u", v);
    else if (offsets[v + 1] - offsets[v] > b->ell)
      bad = fail(RASP_EINVAL, "input of VM %u has %llu words > l = %u", v,
                 (unsigned long long)(offsets[v + 1] - offsets[v]), b->ell);
  }
  if (bad) {
    cudaStreamSynchronize(st);   // the caller's buffers are read before the call returns
    return bad;
  }
  if (b->ellp && !regular) {
    std::vector<uint64_t> buf((size_t)b->V * b->ellp, 0);
    for (uint32_t v = 0; v < b->V; ++v)
      for (uint64_t k = offsets[v]; k < offsets[v + 1]; ++k)
        buf[(size_t)v * b->ellp + (k - offsets[v])] = (uint64_t)tape[k] & b->wmask;
    CK(cudaMemcpyAsync(d_tape, buf.data(), 8 * buf.size(), cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));
  }
  b->max_cap = ~0ull;
  if (caps) {
    uint64_t mx = caps[0];
    bool uniform = true;
    for (uint32_t v = 1; v < b->V; ++v) {
      mx = std::max(mx, caps[v]);
      uniform = uniform && caps[v] == caps[0];
    }
    b->max_cap = mx;
    if (uniform) b->h_caps.clear();
    else b->h_caps.assign(caps, caps + b->V);
  } else {
    CK(fill_bytes(b->d_cap, 0xff, 8ull * b->V, st));
    b->h_caps.clear();
  }
  CK(cudaStreamSynchronize(st));   // the caller's buffers are read before the call returns
  {
    const int rc = order_ids(b);
    if (rc) return rc;
  }
  b->uhead_pending = true;         // u_0 = 0: by the next pack, or before u_0 is next read
  b->inputs_loaded = true;
  g_err.clear();
  return RASP_OK;
}

int rasp_reset(rasp_batch* b) {
  if (!b) return fail(RASP_EINVAL, "batch is NULL");
  if (!b->programs_loaded || !b->inputs_loaded) return fail(RASP_ESTATE, "load programs and inputs first");
  CK(cudaMemsetAsync(b->d_hist, 0, 8 * 10, b->stream));
  b->code_lazy = pack_lazy(b);
  CK(launch_pack(b->S, b->d_prog, b->prog32, b->d_progoff, b->shared_programs ? b->d_progvm : nullptr, b->V,
                 b->wmask, b->sp, b->code_lazy, b->stream));
  b->uhead_pending = false;
  b->dirty_valid = true;
  return RASP_OK;
}

}  // extern "C"

namespace {

// Budget rounds of the HBM-slab persistent schedule. Round r stops every VM
// at min(budget_r, its cap); budgets grow geometrically from kRound0, and the
// last round has the caller's budget (a VM's steps are cumulative, so the
// rounds together equal one run to that budget). Between rounds the VMs of
// the launch group that are still RUNNING are compacted into a dense queue:
// the few long-running VMs then fill whole warps instead of each keeping a
// warp busy whose other lanes have nothing left to run. Rounds are used for
// launch groups larger than the resident lanes (whose lanes are refilled
// from the queue, so that the survivors end up scattered), or always with
// RASP_BUDGET_ROUNDS; a group that fits the resident lanes runs in one launch,
// which also lets concurrent batches (the serving pool) share the GPU without
// waiting for SMs at every round.
constexpr uint64_t kRound0 = 4096;
constexpr uint64_t kRoundGrowth = 8;
constexpr int kMaxRounds = 6;

// Enqueue one rasp_run on `st`: reset the queue counters, one launch per group
// (per budget round for the HBM-slab persistent schedule).
int enqueue_run(rasp_batch* b, cudaStream_t st, uint64_t max_steps) {
  const StepVariant var = variant_of(b);
  Params P{};
  P.wmask = b->wmask;
  P.budget = max_steps;
  P.ell = b->ell;
  P.s = b->s;
  P.ellp = b->ellp;
  P.sp = b->sp;
  P.err = b->d_err;
  P.hist = b->d_hist;
  CK(cudaMemsetAsync(b->d_heads, 0, 8 * kNumBuckets, st));
  uint64_t launches = 0;
  for (size_t k = 0; k < b->groups.size(); ++k) {
    const Group& g = b->groups[k];
    const uint32_t* ids = b->d_ids + g.first;
    if (g.sched != RASP_SCHED_SHARED && b->code_lazy) {
      CK(materialize(b, st));                // these kernels read every word from the slabs
      launches++;
    }
    if (g.sched == RASP_SCHED_SHARED) {
      if (!b->dirty_valid) {
        // another schedule ran since c_0 and did not track code writes: every
        // VM fetches from its own slab until the next reset
        CK(cudaMemsetAsync(b->S.codedirty, 1, b->V, st));
        b->dirty_valid = true;
      }
      CK(ensure_prog64(b, st));
      CK(launch_shared(var, b->S, P, b->d_prog, b->d_progoff, b->d_pvoff, b->d_pvids, b->num_programs,
                       b->max_plen, b->cfg.epoch, st));
    } else if (g.sched == RASP_SCHED_PLAIN) {
      b->dirty_valid = false;
      CK(launch_plain(var, b->S, P, ids, g.count, st));
    } else if (g.sched == RASP_SCHED_PERSIST) {
      b->dirty_valid = false;
      Queue Q{ids, g.count, b->d_heads + k, b->d_heads + kNumBuckets + k, 0, nullptr};
      CK(launch_persist(var, b->S, P, Q, g.shape, st));
    } else {
      b->dirty_valid = false;
      std::vector<uint64_t> budgets;
      const uint64_t limit = std::min(max_steps, b->max_cap);
      const uint64_t lanes = (uint64_t)g.shape.grid * g.shape.warps * 32u;
      const bool rounds = (b->cfg.flags & RASP_BUDGET_ROUNDS) || g.count > lanes;
      for (uint64_t r = kRound0; rounds && r < limit && (int)budgets.size() < kMaxRounds; r *= kRoundGrowth)
        budgets.push_back(r);
      budgets.push_back(max_steps);
      for (size_t r = 0; r < budgets.size(); ++r) {
        uint32_t* head = b->d_heads + k;
        uint32_t* tail = b->d_heads + kNumBuckets + k;
        P.budget = budgets[r];
        if (r == 0) {
          Queue Q{ids, g.count, head, tail, 0, nullptr};
          CK(launch_persist(var, b->S, P, Q, g.shape, st));
        } else {
          uint32_t* dense = b->d_ids2 + g.first;
          CK(launch_compact(ids, g.count, b->S.status, dense, b->d_rcount + k, st));
          CK(cudaMemsetAsync(head, 0, sizeof(uint32_t), st));
          CK(cudaMemsetAsync(tail, 0, sizeof(uint32_t), st));
          Queue Q{dense, g.count, head, tail, 0, b->d_rcount + k};
          CK(launch_persist(var, b->S, P, Q, g.shape, st));
          launches++;                      // the compaction kernel
        }
        launches++;
      }
      P.budget = max_steps;
      continue;
    }
    launches++;
  }
  b->launches = launches;
  return RASP_OK;
}

}  // namespace

extern "C" {

int rasp_run(rasp_batch* b, uint64_t max_steps) {
  if (!b) return fail(RASP_EINVAL, "batch is NULL");
  if (!b->programs_loaded || !b->inputs_loaded) return fail(RASP_ESTATE, "load programs and inputs before rasp_run");
  CK(apply_uhead_reset(b, b->stream));   // eagerly, outside any captured graph
  if (!b->planned) {
    b->planned = true;
    const int rc = replan(b);
    if (rc) return rc;
  }
  // 8-byte program words for the kernels that read them, eagerly (outside any captured graph)
  if (b->code_lazy || (b->cfg.flags & RASP_SCHED_MASK) == RASP_SCHED_SHARED) CK(ensure_prog64(b, b->stream));
  if (!b->cap_stream) return enqueue_run(b, b->stream, max_steps);
  // CUDA graph: capture the run once per budget on a private stream, replay it on the batch stream
  cudaGraphExec_t exec = nullptr;
  for (auto& e : b->graphs)
    if (e.first == max_steps) exec = e.second;
  if (!exec) {
    CK(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
    const int rc = enqueue_run(b, b->cap_stream, max_steps);
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(b->cap_stream, &graph);
    if (rc != RASP_OK) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    if (e != cudaSuccess) return fail(RASP_ECUDA, "cudaStreamEndCapture: %s", cudaGetErrorString(e));
    const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) return fail(RASP_ECUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(ei));
    if (b->graphs.size() >= 8) {
      cudaGraphExecDestroy(b->graphs.front().second);
      b->graphs.erase(b->graphs.begin());
    }
    b->graphs.emplace_back(max_steps, exec);
  }
  CK(cudaGraphLaunch(exec, b->stream));
  return RASP_OK;
}

int rasp_sync(rasp_batch* b) {
  if (!b) return fail(RASP_EINVAL, "batch is NULL");
  return check_device_error(b);
}

int rasp_read_state(rasp_batch* b, uint64_t first, uint64_t count, rasp_state_view* out) {
  if (!b || !out) return fail(RASP_EINVAL, "batch or view is NULL");
  if (first > b->V || count > b->V - first) return fail(RASP_EINVAL, "range [%llu, +%llu) outside the batch",
                                                      (unsigned long long)first, (unsigned long long)count);
  CK(apply_uhead_reset(b, b->stream));
  int rc = check_device_error(b);
  if (rc) return rc;
  if (!count) return RASP_OK;
  cudaStream_t st = b->stream;
  const DevState& S = b->S;
  if (out->i) CK(cudaMemcpyAsync(out->i, S.i + first, 8 * count, cudaMemcpyDeviceToHost, st));
  if (out->a) CK(cudaMemcpyAsync(out->a, S.a + first, 8 * count, cudaMemcpyDeviceToHost, st));
  if (out->steps) CK(cudaMemcpyAsync(out->steps, S.steps + first, 8 * count, cudaMemcpyDeviceToHost, st));
  if (out->status) CK(cudaMemcpyAsync(out->status, S.status + first, count, cudaMemcpyDeviceToHost, st));
  if (out->uhead) CK(cudaMemcpyAsync(out->uhead, S.uhead + first, 4 * count, cudaMemcpyDeviceToHost, st));
  if (out->ylen) CK(cudaMemcpyAsync(out->ylen, S.ylen + first, 4 * count, cudaMemcpyDeviceToHost, st));
  std::vector<uint64_t> ybuf, mbuf;
  std::vector<uint32_t> m32;
  if (out->y && b->s) {
    if (b->sp == b->s) {
      CK(cudaMemcpyAsync(out->y, S.y + first * b->sp, 8 * count * b->sp, cudaMemcpyDeviceToHost, st));
    } else {
      ybuf.resize(count * b->sp);
      CK(cudaMemcpyAsync(ybuf.data(), S.y + first * b->sp, 8 * count * b->sp, cudaMemcpyDeviceToHost, st));
    }
  }
  uint64_t need = 0;
  if (out->mem) CK(materialize(b, st));      // a lazily packed batch: program words into the slabs first
  if (out->mem) {
    for (uint64_t v = first; v < first + count; ++v) need += b->h_n[v];
    if (out->mem_words < need) return fail(RASP_EINVAL, "mem holds %llu words, the range needs %llu",
                                           (unsigned long long)out->mem_words, (unsigned long long)need);
    const uint64_t lo = b->h_memoff[first];
    const uint64_t hi = b->h_memoff[first + count - 1] + even(b->h_n[first + count - 1]);
    if (b->narrow) {                         // 4-byte words, widened below
      m32.resize(hi - lo);
      CK(cudaMemcpyAsync(m32.data(), S.mem32 + lo, 4 * (hi - lo), cudaMemcpyDeviceToHost, st));
    } else if (need == hi - lo) {
      CK(cudaMemcpyAsync(out->mem, S.mem + lo, 8 * need, cudaMemcpyDeviceToHost, st));
    } else {
      mbuf.resize(hi - lo);
      CK(cudaMemcpyAsync(mbuf.data(), S.mem + lo, 8 * (hi - lo), cudaMemcpyDeviceToHost, st));
    }
  }
  CK(cudaStreamSynchronize(st));
  if (!ybuf.empty())
    for (uint64_t v = 0; v < count; ++v)
      memcpy(out->y + v * b->s, ybuf.data() + v * b->sp, 8 * b->s);
  if (!mbuf.empty()) {
    const uint64_t lo = b->h_memoff[first];
    uint64_t o = 0;
    for (uint64_t v = first; v < first + count; ++v) {
      memcpy(out->mem + o, mbuf.data() + (b->h_memoff[v] - lo), 8ull * b->h_n[v]);
      o += b->h_n[v];
    }
  }
  if (!m32.empty()) {
    const uint64_t lo = b->h_memoff[first];
    uint64_t o = 0;
    for (uint64_t v = first; v < first + count; ++v) {
      const uint32_t* src = m32.data() + (b->h_memoff[v] - lo);
      for (uint32_t k = 0; k < b->h_n[v]; ++k) out->mem[o + k] = (int64_t)src[k];
      o += b->h_n[v];
    }
  }
  return RASP_OK;
}

int rasp_load_state(rasp_batch* b, uint64_t first, uint64_t count, const rasp_state_view* in) {
  if (!b || !in) return fail(RASP_EINVAL, "batch or view is NULL");
  if (first > b->V || count > b->V - first) return fail(RASP_EINVAL, "range outside the batch");
  if (!count) return RASP_OK;
  for (uint64_t v = 0; v < count; ++v) {
    if (in->uhead && in->uhead[v] > b->ell) return fail(RASP_EINVAL, "u_0 of VM %llu exceeds l", (unsigned long long)(first + v));
    if (in->ylen && in->ylen[v] > b->s) return fail(RASP_EINVAL, "y_0 of VM %llu exceeds s", (unsigned long long)(first + v));
    if (in->status && in->status[v] > RASP_FAULT_ADDR) return fail(RASP_EINVAL, "bad status for VM %llu", (unsigned long long)(first + v));
  }
  uint64_t need = 0;
  if (in->mem) {
    for (uint64_t v = first; v < first + count; ++v) need += b->h_n[v];
    if (in->mem_words < need) return fail(RASP_EINVAL, "mem holds %llu words, the range needs %llu",
                                          (unsigned long long)in->mem_words, (unsigned long long)need);
  }
  cudaStream_t st = b->stream;
  const DevState& S = b->S;
  CK(apply_uhead_reset(b, st));
  if (in->i) CK(cudaMemcpyAsync(S.i + first, in->i, 8 * count, cudaMemcpyHostToDevice, st));
  if (in->a) CK(cudaMemcpyAsync(S.a + first, in->a, 8 * count, cudaMemcpyHostToDevice, st));
  if (in->steps) CK(cudaMemcpyAsync(S.steps + first, in->steps, 8 * count, cudaMemcpyHostToDevice, st));
  if (in->status) CK(cudaMemcpyAsync(S.status + first, in->status, count, cudaMemcpyHostToDevice, st));
  if (in->uhead) CK(cudaMemcpyAsync(S.uhead + first, in->uhead, 4 * count, cudaMemcpyHostToDevice, st));
  if (in->ylen) CK(cudaMemcpyAsync(S.ylen + first, in->ylen, 4 * count, cudaMemcpyHostToDevice, st));
  std::vector<uint64_t> ybuf, mbuf;
  if (in->y && b->s) {
    ybuf.assign(count * b->sp, 0);
    for (uint64_t v = 0; v < count; ++v)
      for (uint32_t k = 0; k < b->s; ++k) ybuf[v * b->sp + k] = (uint64_t)in->y[v * b->s + k] & b->wmask;
    CK(cudaMemcpyAsync(S.y + first * b->sp, ybuf.data(), 8 * ybuf.size(), cudaMemcpyHostToDevice, st));
  }
  std::vector<uint32_t> m32;
  if (in->mem) {
    const uint64_t lo = b->h_memoff[first];
    const uint64_t hi = b->h_memoff[first + count - 1] + even(b->h_n[first + count - 1]);
    if (b->narrow) m32.assign(hi - lo, 0);
    else mbuf.assign(hi - lo, 0);
    uint64_t o = 0;
    for (uint64_t v = first; v < first + count; ++v) {
      for (uint32_t k = 0; k < b->h_n[v]; ++k) {
        const uint64_t w = (uint64_t)in->mem[o + k] & b->wmask;
        if (b->narrow) m32[b->h_memoff[v] - lo + k] = (uint32_t)w;
        else mbuf[b->h_memoff[v] - lo + k] = w;
      }
      o += b->h_n[v];
    }
    if (b->narrow) CK(cudaMemcpyAsync(S.mem32 + lo, m32.data(), 4 * m32.size(), cudaMemcpyHostToDevice, st));
    else CK(cudaMemcpyAsync(S.mem + lo, mbuf.data(), 8 * mbuf.size(), cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(b->S.codedirty + first, 1, count, st));   // restored M may differ from the program
  }
  CK(cudaStreamSynchronize(st));
  return RASP_OK;
}

int rasp_halting_histogram(rasp_batch* b, const uint64_t* edges, uint32_t nbins, uint64_t* counts,
                           uint64_t* other) {
  if (!b || !edges || !counts) return fail(RASP_EINVAL, "batch, edges or counts is NULL");
  if (nbins == 0 || nbins > kMaxHistBins) return fail(RASP_EINVAL, "nbins must be in 1..%u", kMaxHistBins);
  for (uint32_t k = 0; k < nbins; ++k)
    if (edges[k] >= edges[k + 1]) return fail(RASP_EINVAL, "edges must increase strictly (edges[%u])", k);
  int rc = check_device_error(b);
  if (rc) return rc;
  cudaStream_t st = b->stream;
  uint64_t* d_edges = (uint64_t*)(b->base + b->L.off_thist);
  unsigned long long* d_counts = (unsigned long long*)(d_edges + kMaxHistBins + 1);
  unsigned long long* d_other = d_counts + kMaxHistBins;
  uint64_t oth[4] = {0, 0, 0, 0};
  CK(cudaMemcpyAsync(d_edges, edges, 8ull * (nbins + 1), cudaMemcpyHostToDevice, st));
  CK(launch_tau_hist(b->S, b->V, d_edges, nbins, d_counts, d_other, st));
  CK(cudaMemcpyAsync(counts, d_counts, 8ull * nbins, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(oth, d_other, sizeof(oth), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (other) memcpy(other, oth, sizeof(oth));
  return RASP_OK;
}

int rasp_top_halting(rasp_batch* b, uint32_t k, uint64_t* steps_out, uint32_t* vm_out, uint32_t* found) {
  if (!b || !steps_out || !vm_out || !found) return fail(RASP_EINVAL, "batch or an output pointer is NULL");
  if (k == 0 || k > kMaxTopK) return fail(RASP_EINVAL, "k must be in 1..%u", kMaxTopK);
  int rc = check_device_error(b);
  if (rc) return rc;
  cudaStream_t st = b->stream;
  TopCand* cand = (TopCand*)(b->base + b->L.off_topk);
  TopCand* best = cand + (size_t)topk_blocks(b->V) * kMaxTopK;
  std::vector<TopCand> h(k);
  CK(launch_topk(b->S, b->V, k, cand, best, st));
  CK(cudaMemcpyAsync(h.data(), best, sizeof(TopCand) * k, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  uint32_t n = 0;
  for (uint32_t q = 0; q < k && h[q].ok; ++q, ++n) {
    steps_out[q] = h[q].steps;
    vm_out[q] = h[q].vm;
  }
  *found = n;
  return RASP_OK;
}

int rasp_read_stats(rasp_batch* b, rasp_stats* out) {
  if (!b || !out) return fail(RASP_EINVAL, "batch or stats is NULL");
  int rc = check_device_error(b);
  if (rc) return rc;
  unsigned long long agg[6] = {0, 0, 0, 0, 0, 0}, hist[10] = {0};
  CK(launch_stats(b->S, b->V, b->d_stats, b->stream));
  CK(cudaMemcpyAsync(agg, b->d_stats, sizeof(agg), cudaMemcpyDeviceToHost, b->stream));
  CK(cudaMemcpyAsync(hist, b->d_hist, sizeof(hist), cudaMemcpyDeviceToHost, b->stream));
  CK(cudaStreamSynchronize(b->stream));
  memset(out, 0, sizeof(*out));
  out->vm_steps = agg[0];
  out->running = agg[1];
  out->halted = agg[2];
  out->timeout = agg[3];
  out->fault_overflow = agg[4];
  out->fault_addr = agg[5];
  for (int k = 1; k <= 7; ++k) out->op_steps[k] = hist[k];
  out->pri_full = hist[8];
  out->bnz_taken = hist[9];
  out->launches = b->launches;
  return RASP_OK;
}

}  // extern "C"

namespace {

void drop_graphs(rasp_batch* b) {
  for (auto& e : b->graphs) cudaGraphExecDestroy(e.second);
  b->graphs.clear();
}

int replan(rasp_batch* b) {
  plan_buckets(b);
  build_groups(b);
  drop_graphs(b);
  return b->inputs_loaded ? order_ids(b) : RASP_OK;
}

}  // namespace

extern "C" {

int rasp_autotune(rasp_batch* b, uint64_t max_steps, uint32_t reps) {
  if (!b) return fail(RASP_EINVAL, "batch is NULL");
  if (!b->programs_loaded || !b->inputs_loaded) return fail(RASP_ESTATE, "load programs and inputs before tuning");
  if (reps == 0) reps = 1;
  CK(apply_uhead_reset(b, b->stream));
  if (b->shared_programs || b->code_lazy) CK(ensure_prog64(b, b->stream));   // the shared-program trials
  int rc = check_device_error(b);
  if (rc) return rc;
  cudaStream_t st = b->stream;
  const Layout& L = b->L;
  // mutable state: i, a, steps | status, uhead, ylen | M | y | counters
  const size_t spans[][2] = {{L.off_i, L.off_cap}, {L.off_status, L.off_n}, {L.off_mem, L.off_prog},
                             {L.off_y, L.off_ids}, {L.off_hist, L.off_stats}, {L.off_dirty, L.off_dirty + b->V}};
  const bool dirty_valid0 = b->dirty_valid, code_lazy0 = b->code_lazy;
  size_t total = 0;
  for (auto& sp : spans) total += sp[1] - sp[0];
  char* snap = nullptr;
  if (inject_alloc_failure() || cudaMalloc(&snap, total) != cudaSuccess) {
    cudaGetLastError();
    return fail(RASP_ENOMEM, "autotune needs %llu bytes for a snapshot of the state", (unsigned long long)total);
  }
  auto copy_state = [&](bool save) -> cudaError_t {
    size_t o = 0;
    for (auto& sp : spans) {
      const size_t len = sp[1] - sp[0];
      cudaError_t e = save ? cudaMemcpyAsync(snap + o, b->base + sp[0], len, cudaMemcpyDeviceToDevice, st)
                           : cudaMemcpyAsync(b->base + sp[0], snap + o, len, cudaMemcpyDeviceToDevice, st);
      if (e != cudaSuccess) return e;
      o += len;
    }
    return cudaSuccess;
  };
  // HBM-slab persistent shapes: epochs, CTA sizes and resident CTAs per SM
  // (fewer resident VMs keep large memories in L1/L2: the uneven batch runs
  // best at 12 warps per SM, the template batch at 28)
  // The SMEM-staged schedule in both forms: its epoch loop, and one step at
  // a time (fastest when a few thousand short runs leave the loop often).
  struct Cand { const char* name; uint32_t sched, epoch, warps, ctas; bool block; };
  static const Cand cands[] = {
      {"persist_gl e128 w4", RASP_SCHED_PERSIST_GL, 128, 4, 0, false},
      {"persist_gl e64 w4", RASP_SCHED_PERSIST_GL, 64, 4, 0, false},
      {"persist_gl e256 w4", RASP_SCHED_PERSIST_GL, 256, 4, 0, false},
      {"persist_gl e128 w2", RASP_SCHED_PERSIST_GL, 128, 2, 0, false},
      {"persist_gl e128 w4 c3", RASP_SCHED_PERSIST_GL, 128, 4, 3, false},
      {"persist_gl e128 w4 c5", RASP_SCHED_PERSIST_GL, 128, 4, 5, false},
      {"plain", RASP_SCHED_PLAIN, 0, 0, 0, false},
      {"persist_smem e128 w1", RASP_SCHED_PERSIST, 128, 1, 0, false},
      {"persist_smem e32 w1 step", RASP_SCHED_PERSIST, 32, 1, 0, true},
      {"shared", RASP_SCHED_SHARED, 0, 0, 0, false}};
  // the shared-program schedule is a candidate only when programs are shared;
  // the classic opcode set runs on the HBM-slab persistent and plain schedules only
  const bool classic = (b->cfg.flags & RASP_ISA_CLASSIC) != 0;
  const int ncand = classic ? 7 : (int)(sizeof(cands) / sizeof(cands[0])) - (b->shared_programs && !b->narrow ? 0 : 1);
  const rasp_config saved = b->cfg;
  b->over.clear();                         // the global pass tunes the batch-wide settings
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaError_t ce = copy_state(true);
  // one timed rasp_run of the current plan (the state put back before each
  // repetition); the fastest repetition
  auto trial = [&](float& tmin) -> int {
    int r2 = replan(b);
    if (r2) return r2;
    tmin = 1e30f;
    for (uint32_t r = 0; r < reps && ce == cudaSuccess; ++r) {
      ce = copy_state(false);
      b->dirty_valid = dirty_valid0;
      b->code_lazy = code_lazy0;
      if (ce != cudaSuccess) break;
      cudaEventRecord(e0, st);
      r2 = enqueue_run(b, st, max_steps);
      if (r2) return r2;
      cudaEventRecord(e1, st);
      ce = cudaEventSynchronize(e1);
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      tmin = std::min(tmin, ms);
    }
    return RASP_OK;
  };
  auto adopt = [&](rasp_config& c, const Cand& k) {
    c.flags = (saved.flags & ~RASP_SCHED_MASK) | k.sched;
    b->tuned_block = k.block;
    c.epoch = k.epoch;
    c.warps_per_cta = k.warps;
    c.ctas_per_sm = k.ctas;
  };
  float best = 1e30f;
  int best_k = -1;
  std::string rep = "{\"budget\": " + std::to_string(max_steps) + ", \"trials\": [";
  for (int k = 0; ce == cudaSuccess && k < ncand; ++k) {
    adopt(b->cfg, cands[k]);
    float tmin = 0;
    rc = trial(tmin);
    if (rc || ce != cudaSuccess) break;
    char tmp[128];
    snprintf(tmp, sizeof(tmp), "%s{\"schedule\": \"%s\", \"ms\": %.4f}", k ? ", " : "", cands[k].name, tmin);
    rep += tmp;
    if (tmin < best) {
      best = tmin;
      best_k = k;
    }
  }
  rep += "]";
  b->cfg = saved;
  b->tuned_block = false;
  if (best_k >= 0) adopt(b->cfg, cands[best_k]);
  // Per-bucket pass (coordinate descent over the memory-size buckets): with
  // every other bucket on its current choice, each bucket tries the other
  // thread-per-VM shapes and keeps one only if the whole run gets faster by
  // more than 1 %. Buckets that end up with different shapes launch
  // separately.
  std::string brep;
  int nonempty = 0;
  for (const Bucket& k : b->buckets) nonempty += k.count ? 1 : 0;
  if (!rc && ce == cudaSuccess && best_k >= 0 && cands[best_k].sched != RASP_SCHED_SHARED && nonempty > 1) {
    b->over.assign(b->buckets.size(), BucketPlan{});
    float cur = best;
    brep = ", \"buckets\": [";
    bool firstb = true;
    for (size_t bi = 0; bi < b->buckets.size() && !rc && ce == cudaSuccess; ++bi) {
      if (!b->buckets[bi].count) continue;
      int chosen = -1;
      std::string tr;
      for (int k = 0; k < ncand && !rc && ce == cudaSuccess; ++k) {
        // other epochs are left to the global pass: per bucket, the shapes
        // that change the schedule or the resident VMs per SM
        if (k == best_k || cands[k].sched == RASP_SCHED_SHARED || cands[k].epoch == 64 || cands[k].epoch == 256)
          continue;
        const BucketPlan keep = b->over[bi];
        b->over[bi] = BucketPlan{true, cands[k].sched, cands[k].epoch, cands[k].warps, cands[k].ctas, cands[k].block};
        float tmin = 0;
        rc = trial(tmin);
        if (rc || ce != cudaSuccess) break;
        char tmp[128];
        snprintf(tmp, sizeof(tmp), "%s{\"schedule\": \"%s\", \"ms\": %.4f}", tr.empty() ? "" : ", ",
                 cands[k].name, tmin);
        tr += tmp;
        if (tmin < cur * 0.99f) {
          cur = tmin;
          chosen = k;
        } else {
          b->over[bi] = keep;
        }
      }
      char tmp[160];
      snprintf(tmp, sizeof(tmp), "%s{\"n_max\": %u, \"chosen\": \"%s\", \"trials\": [", firstb ? "" : ", ",
               b->buckets[bi].ncap, chosen >= 0 ? cands[chosen].name : cands[best_k].name);
      brep += tmp + tr + "]}";
      firstb = false;
    }
    brep += "]";
    bool any = false;
    for (const BucketPlan& o : b->over) any = any || o.set;
    if (!any) b->over.clear();
    char tmp[64];
    snprintf(tmp, sizeof(tmp), ", \"per_bucket_ms\": %.4f", cur);
    brep += tmp;
  }
  // leave the state as it was, with the chosen plan
  const cudaError_t ce2 = copy_state(false);
  b->dirty_valid = dirty_valid0;
  b->code_lazy = code_lazy0;
  cudaStreamSynchronize(st);
  cudaFree(snap);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc || ce != cudaSuccess) b->over.clear();
  const int rc2 = replan(b);
  if (rc) return rc;
  if (rc2) return rc2;
  if (ce != cudaSuccess || ce2 != cudaSuccess)
    return fail(RASP_ECUDA, "autotune: %s", cudaGetErrorString(ce != cudaSuccess ? ce : ce2));
  rep += ", \"chosen\": \"";
  rep += best_k >= 0 ? cands[best_k].name : "none";
  rep += "\"";
  rep += brep;
  rep += "}";
  b->tuned = rep;
  return check_device_error(b);
}

int rasp_plan_bucket(rasp_batch* b, uint32_t bucket, uint32_t sched, uint32_t epoch, uint32_t warps_per_cta,
                     uint32_t ctas_per_sm) {
  if (!b) return fail(RASP_EINVAL, "batch is NULL");
  if (bucket >= b->buckets.size()) return fail(RASP_EINVAL, "bucket %u out of range (%zu buckets)", bucket,
                                               b->buckets.size());
  if (sched != RASP_SCHED_AUTO && sched != RASP_SCHED_PLAIN && sched != RASP_SCHED_PERSIST &&
      sched != RASP_SCHED_PERSIST_GL)
    return fail(RASP_EINVAL, "per-bucket schedule must be AUTO, PLAIN, PERSIST or PERSIST_GL");
  if ((b->cfg.flags & RASP_SCHED_MASK) == RASP_SCHED_SHARED)
    return fail(RASP_EINVAL, "the shared-program schedule runs all buckets in one launch");
  if ((b->cfg.flags & RASP_ISA_CLASSIC) && sched == RASP_SCHED_PERSIST)
    return fail(RASP_EINVAL, "the classic opcode set runs on the plain and HBM-slab persistent schedules only");
  if (b->over.size() != b->buckets.size()) b->over.assign(b->buckets.size(), BucketPlan{});
  b->over[bucket] = BucketPlan{sched != RASP_SCHED_AUTO, sched, epoch, warps_per_cta, ctas_per_sm};
  if (!b->planned) return RASP_OK;       // planned at the first rasp_run
  return replan(b);
}

int rasp_describe(const rasp_batch* b, char* buf, uint64_t size) {
  if (!b || !buf || size == 0) return fail(RASP_EINVAL, "batch or buffer is NULL");
  static const char* names[] = {"auto", "plain", "persist", "persist_gl", "shared"};
  std::string s = "{\"vms\": " + std::to_string(b->V) + ", \"buckets\": [";
  bool first = true;
  for (size_t bi = 0; bi < b->buckets.size(); ++bi) {
    const Bucket& k = b->buckets[bi];
    if (!k.count) continue;
    char tmp[512];
    snprintf(tmp, sizeof(tmp),
             "%s{\"index\": %zu, \"n_max\": %u, \"vms\": %u, \"schedule\": \"%s\", \"grid\": %u, "
             "\"warps_per_cta\": %u, \"ctas_per_sm\": %u, \"smem\": %zu, \"epoch\": %u, \"refill_min\": %u, "
             "\"pinned\": %s}",
             first ? "" : ", ", bi, k.ncap, k.count, names[std::min<uint32_t>(k.sched >> 4, 4u)], k.shape.grid, k.shape.warps,
             k.shape.ctas_per_sm, k.shape.smem, k.shape.epoch, k.shape.refill_min,
             (bi < b->over.size() && b->over[bi].set) ? "true" : "false");
    s += tmp;
    first = false;
  }
  s += "], \"launches\": [";
  first = true;
  for (const Group& g : b->groups) {
    char tmp[256];
    snprintf(tmp, sizeof(tmp), "%s{\"vms\": %u, \"schedule\": \"%s\", \"grid\": %u}", first ? "" : ", ",
             g.count, names[std::min<uint32_t>(g.sched >> 4, 4u)], g.shape.grid);
    s += tmp;
    first = false;
  }
  s += "], \"word_bytes\": ";
  s += b->narrow ? "4" : "8";
  s += ", \"program_word_bytes\": ";      // how the pack reads the loaded programs
  s += b->prog32 ? "4" : "8";
  s += ", \"cuda_graph\": ";
  s += b->cap_stream ? "true" : "false";
  s += ", \"autotune\": ";
  s += b->tuned.empty() ? "null" : b->tuned;
  s += "}";
  if (s.size() + 1 > size) return fail(RASP_EINVAL, "buffer of %llu bytes is too small", (unsigned long long)size);
  memcpy(buf, s.c_str(), s.size() + 1);
  return RASP_OK;
}

void rasp_batch_destroy(rasp_batch* b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  for (auto& e : b->graphs) cudaGraphExecDestroy(e.second);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  if (b->owns && b->base) cudaFree(b->base);
  delete b;
}

}  // extern "C"
