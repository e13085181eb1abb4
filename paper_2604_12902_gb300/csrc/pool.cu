// pool.cu -- serving: continuous batching of rollout requests.
//
// A pool owns one device arena. A submitted request (programs, tapes, caps,
// memory sizes) is admitted as soon as a first-fit block of the arena, a
// request slot and room on the ring can hold it; it then gets its own batch
// carved from that block (its state store, loaded and packed to c_0 on its
// own stream). Admission puts one entry per VM -- (slot, VM) -- on a ring in
// device memory that all admitted requests share, and publishes the new tail.
// One persistent serving kernel (k_serve) drains the ring: its lanes take the
// next entries as their VMs stop, whichever request they belong to, so work
// that arrives while other requests run fills the lanes those requests free
// (continuous batching of lanes, not only of memory). The lane that stops a
// request's last VM writes the request's completion word in host-mapped
// memory, which poll/next_done read without a CUDA call. Requests that do
// not fit wait first-in-first-out; reading a result frees its block and slot
// and admits waiting requests.
//
// Ordering: a request's loads run on its stream; the ring stream waits for
// them, writes the request's slot descriptor and its ring entries, and then
// publishes them (adds their count to the claimable credits); the run
// stream waits for the publish and launches a serving kernel instance. An
// instance returns as a whole once the ring is empty and none of its warps
// holds work -- at once if the host has launched a newer instance (ordered
// after every later publish), else after a bounded idle wait -- so every
// published VM is run by some instance and no kernel waits on the host
// without a limit.
#include <chrono>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/rasp.h"
#include "internal.h"

using namespace rasp;

namespace {

thread_local std::string g_pool_err;

int pfail(int code, const std::string& msg) {
  g_pool_err = msg;
  return code;
}

constexpr uint32_t kMaxSlots = 1024;             // requests admitted at once
constexpr uint64_t kRingCap = 1ull << 24;        // VMs admitted and not yet read (ring entries)
constexpr uint32_t kIdlePolls = 200;             // about 3 ms of empty ring before the newest instance returns

struct Request {
  uint64_t ticket = 0;
  int state = RASP_REQ_QUEUED;
  uint64_t num_vms = 0;
  // host copies of the inputs while the request waits for admission (a
  // request admitted at submit is loaded from the caller's buffers instead)
  std::vector<int64_t> words, tape;
  std::vector<uint64_t> offsets, tape_off, caps;
  std::vector<uint32_t> prog_of_vm, mem_words;
  uint64_t num_programs = 0;
  uint64_t max_steps = 0;
  bool has_caps = false;
  // admitted
  uint64_t bytes = 0, offset = 0;
  rasp_batch* batch = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t loaded = nullptr;
  uint32_t slot = ~0u;
  uint32_t gen = 0;
  bool on_ring = false;
  int error = RASP_OK;
  std::string error_msg;
};

}  // namespace

struct rasp_pool {
  rasp_config cfg{};
  char* base = nullptr;
  uint64_t bytes = 0;
  std::map<uint64_t, uint64_t> free_blocks;   // offset -> size
  std::map<uint64_t, Request> reqs;
  std::deque<uint64_t> waiting;
  uint64_t next_ticket = 1;
  uint64_t in_use = 0;
  std::deque<uint64_t> done;                  // finished, not yet handed out by rasp_pool_next_done
  std::mutex mu;
  // the serving ring and its kernel
  StepVariant var{};
  ServeShape shape{};
  uint32_t epoch = 128;
  cudaStream_t ring_stream = nullptr, run_stream = nullptr;
  cudaEvent_t published = nullptr;
  char* dev = nullptr;                        // slots | pending | ring | head, credits, state
  ServeSlot* d_slots = nullptr;
  uint32_t* d_pending = nullptr;
  uint64_t* d_ring = nullptr;
  unsigned long long* d_head = nullptr;
  unsigned long long* d_credits = nullptr;
  unsigned long long* d_state = nullptr;
  char* pinned = nullptr;                     // staging of slot descriptors and counts
  ServeSlot* h_slots = nullptr;
  uint32_t* h_pending = nullptr;
  uint32_t* mapped = nullptr;                 // host-mapped: done[kMaxSlots] | launched | exited | err
  uint32_t* d_mapped = nullptr;
  std::vector<uint32_t> free_slots;
  std::vector<std::pair<cudaStream_t, cudaEvent_t>> spare;   // of retired requests
  unsigned long long tail = 0;                // published positions
  uint64_t ring_used = 0;                     // VMs admitted and not yet read
  uint32_t launches = 0;
  uint64_t admitted = 0, completed = 0;
};

namespace {

constexpr uint64_t kAlign = 256;

volatile uint32_t* done_word(rasp_pool* p, uint32_t slot) { return p->mapped + slot; }
volatile uint32_t* launched_word(rasp_pool* p) { return p->mapped + kMaxSlots; }
volatile uint32_t* exited_word(rasp_pool* p) { return p->mapped + kMaxSlots + 1; }
volatile uint32_t* err_word(rasp_pool* p) { return p->mapped + kMaxSlots + 2; }

bool carve(rasp_pool* p, uint64_t need, uint64_t* off) {
  for (auto it = p->free_blocks.begin(); it != p->free_blocks.end(); ++it) {
    if (it->second >= need) {
      *off = it->first;
      const uint64_t rest = it->second - need;
      const uint64_t roff = it->first + need;
      p->free_blocks.erase(it);
      if (rest) p->free_blocks[roff] = rest;
      p->in_use += need;
      return true;
    }
  }
  return false;
}

void release(rasp_pool* p, uint64_t off, uint64_t size) {
  p->in_use -= size;
  auto it = p->free_blocks.emplace(off, size).first;
  auto nx = std::next(it);
  if (nx != p->free_blocks.end() && it->first + it->second == nx->first) {
    it->second += nx->second;
    p->free_blocks.erase(nx);
  }
  if (it != p->free_blocks.begin()) {
    auto pv = std::prev(it);
    if (pv->first + pv->second == it->first) {
      pv->second += it->second;
      p->free_blocks.erase(it);
    }
  }
}

// Room for one more request of `vms` VMs in `need` bytes: a slot, ring room
// and (first fit) arena memory, carved if there is.
bool reserve(rasp_pool* p, uint64_t vms, uint64_t need, uint64_t* off) {
  if (p->free_slots.empty() || p->ring_used + vms > kRingCap) return false;
  return carve(p, need, off);
}

void fail_request(Request& r, int code, const char* where) {
  r.state = RASP_REQ_DONE;
  r.error = code;
  r.error_msg = std::string(where) + ": " + rasp_last_error();
}

// Put the admitted, loaded request on the ring and make sure a serving
// kernel instance runs after it is published.
int publish(rasp_pool* p, Request& r) {
  const uint32_t slot = p->free_slots.back();
  p->free_slots.pop_back();
  r.slot = slot;
  r.gen = (uint32_t)(r.ticket & 0x7FFFFFFFu) | 0x80000000u;   // nonzero
  *done_word(p, slot) = 0u;
  ServeSlot& hs = p->h_slots[slot];
  hs.S = batch_dev_state(r.batch);
  hs.budget = r.max_steps;
  hs.num_vms = (uint32_t)r.num_vms;
  hs.gen = r.gen;
  p->h_pending[slot] = (uint32_t)r.num_vms;
  cudaStream_t rs = p->ring_stream;
  if (cudaStreamWaitEvent(rs, r.loaded, 0) != cudaSuccess ||
      cudaMemcpyAsync(p->d_slots + slot, &hs, sizeof(ServeSlot), cudaMemcpyHostToDevice, rs) != cudaSuccess ||
      cudaMemcpyAsync(p->d_pending + slot, p->h_pending + slot, sizeof(uint32_t), cudaMemcpyHostToDevice, rs) !=
          cudaSuccess ||
      launch_ring_append(p->d_ring, kRingCap - 1, p->tail, slot, batch_queue(r.batch), (uint32_t)r.num_vms,
                         p->d_credits, rs) != cudaSuccess ||
      cudaEventRecord(p->published, rs) != cudaSuccess || cudaStreamWaitEvent(p->run_stream, p->published, 0) != cudaSuccess) {
    cudaGetLastError();
    p->free_slots.push_back(slot);
    r.slot = ~0u;
    return RASP_ECUDA;
  }
  p->tail += r.num_vms;
  p->ring_used += r.num_vms;
  r.on_ring = true;
  // a new instance, ordered after this publish; the running one sees the
  // newer count and returns as soon as the ring is empty
  ServeArgs A{};
  A.slots = p->d_slots;
  A.num_slots = kMaxSlots;
  A.pending = p->d_pending;
  A.ring = p->d_ring;
  A.ring_mask = kRingCap - 1;
  A.head = p->d_head;
  A.credits = p->d_credits;
  A.state = p->d_state;
  A.done = p->d_mapped;
  A.launched = p->d_mapped + kMaxSlots;
  A.exited = p->d_mapped + kMaxSlots + 1;
  A.instance = p->launches + 1;
  A.epoch = p->epoch;
  A.idle_polls = kIdlePolls;
  A.err = reinterpret_cast<int*>(p->d_mapped + kMaxSlots + 2);
  Params P = batch_params(r.batch);
  P.err = A.err;
  P.hist = nullptr;
  if (cudaMemsetAsync(p->d_state, 0, sizeof(unsigned long long), p->run_stream) != cudaSuccess ||
      launch_serve(p->var, A, P, p->shape, p->run_stream) != cudaSuccess) {
    cudaGetLastError();
    return RASP_ECUDA;
  }
  p->launches = A.instance;
  *launched_word(p) = p->launches;
  p->admitted++;
  return RASP_OK;
}

// Start one admitted request from the host inputs `q`: batch in its block,
// own stream, loads, then onto the ring.
void start(rasp_pool* p, Request& r, const rasp_request& q) {
  rasp_config c = p->cfg;
  c.arena = p->base + r.offset;
  c.arena_bytes = r.bytes;
  c.flags &= ~RASP_CUDA_GRAPH;
  if (!p->spare.empty()) {                    // streams and events are reused across requests
    r.stream = p->spare.back().first;
    r.loaded = p->spare.back().second;
    p->spare.pop_back();
  } else if (cudaStreamCreateWithFlags(&r.stream, cudaStreamNonBlocking) != cudaSuccess ||
             cudaEventCreateWithFlags(&r.loaded, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    r.state = RASP_REQ_DONE;
    r.error = RASP_ECUDA;
    r.error_msg = "cannot create a stream or event";
    return;
  }
  c.stream = r.stream;
  int rc = create_batch(&c, q.num_vms, q.mem_words, false, &r.batch);
  if (rc) return fail_request(r, rc, "create");
  // inputs first: each load waits until it has read the caller's buffers,
  // and the program load ends by launching the c_0 pack without waiting for
  // it, so the host never waits for a pack that runs beside the serving kernel
  rc = rasp_load_inputs(r.batch, q.tape, q.tape_off, q.caps);
  if (rc) return fail_request(r, rc, "load_inputs");
  rc = rasp_load_programs(r.batch, q.words, q.offsets, q.num_programs, q.prog_of_vm);
  if (rc) return fail_request(r, rc, "load_programs");
  if (cudaEventRecord(r.loaded, r.stream) != cudaSuccess) {
    cudaGetLastError();
    r.state = RASP_REQ_DONE;
    r.error = RASP_ECUDA;
    r.error_msg = "cannot record the load event";
    return;
  }
  rc = publish(p, r);
  if (rc) {
    r.state = RASP_REQ_DONE;
    r.error = rc;
    r.error_msg = "cannot put the request on the ring";
    return;
  }
  r.state = RASP_REQ_RUNNING;
  // inputs are on the device now
  std::vector<uint32_t>().swap(r.mem_words);
  std::vector<int64_t>().swap(r.words);
  std::vector<int64_t>().swap(r.tape);
  std::vector<uint64_t>().swap(r.offsets);
  std::vector<uint64_t>().swap(r.tape_off);
  std::vector<uint64_t>().swap(r.caps);
  std::vector<uint32_t>().swap(r.prog_of_vm);
}

// The host inputs held by a waiting request.
rasp_request held_inputs(const Request& r) {
  rasp_request q{};
  q.words = r.words.data();
  q.offsets = r.offsets.data();
  q.num_programs = r.num_programs;
  q.prog_of_vm = r.prog_of_vm.empty() ? nullptr : r.prog_of_vm.data();
  q.tape = r.tape.data();
  q.tape_off = r.tape_off.data();
  q.caps = r.has_caps ? r.caps.data() : nullptr;
  q.mem_words = r.mem_words.data();
  q.num_vms = r.num_vms;
  q.max_steps = r.max_steps;
  return q;
}

// Admit waiting requests in arrival order while there is room.
void admit(rasp_pool* p) {
  while (!p->waiting.empty()) {
    Request& r = p->reqs[p->waiting.front()];
    uint64_t off = 0;
    if (!reserve(p, r.num_vms, r.bytes, &off)) break;
    r.offset = off;
    p->waiting.pop_front();
    start(p, r, held_inputs(r));
    if (r.state == RASP_REQ_DONE) p->done.push_back(r.ticket);   // failed at admission
  }
}

// A running request whose completion word is set is DONE.
bool check_done(rasp_pool* p, Request& r) {
  if (r.state != RASP_REQ_RUNNING) return false;
  if (*done_word(p, r.slot) != r.gen) return false;
  r.state = RASP_REQ_DONE;
  return true;
}

// Every serving kernel instance launched so far has returned (each of its
// CTAs adds one to the exited word; counted modulo 2^32).
bool kernels_idle(rasp_pool* p) {
  return *exited_word(p) == (uint32_t)((uint64_t)p->launches * p->shape.grid);
}

// Wait for a running request's completion word. If every launched instance
// has returned and the word is still not set, the request cannot finish: the
// wait ends with RASP_EDEVICE instead of waiting forever.
int wait_done(rasp_pool* p, Request& r) {
  while (r.state == RASP_REQ_RUNNING) {
    if (check_done(p, r)) break;
    if (kernels_idle(p)) {
      if (check_done(p, r)) break;
      return RASP_EDEVICE;
    }
    std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
  return RASP_OK;
}

int device_error(rasp_pool* p) { return *err_word(p) ? RASP_EDEVICE : RASP_OK; }

// Free an admitted request's resources (its VMs are no longer on the ring).
void retire(rasp_pool* p, Request& r) {
  if (r.batch) rasp_batch_destroy(r.batch);      // waits for the request's stream
  else if (r.stream) cudaStreamSynchronize(r.stream);
  if (r.stream && r.loaded) {
    p->spare.emplace_back(r.stream, r.loaded);
  } else {
    if (r.loaded) cudaEventDestroy(r.loaded);
    if (r.stream) cudaStreamDestroy(r.stream);
  }
  r.batch = nullptr;
  r.loaded = nullptr;
  r.stream = nullptr;
  if (r.slot != ~0u) {
    p->free_slots.push_back(r.slot);
    r.slot = ~0u;
  }
  if (r.on_ring) {
    p->ring_used -= r.num_vms;
    r.on_ring = false;
  }
  if (r.state != RASP_REQ_QUEUED) release(p, r.offset, r.bytes);
}

void free_pool(rasp_pool* p) {
  if (p->run_stream) cudaStreamSynchronize(p->run_stream);
  if (p->ring_stream) cudaStreamSynchronize(p->ring_stream);
  if (p->published) cudaEventDestroy(p->published);
  for (auto& se : p->spare) {
    cudaEventDestroy(se.second);
    cudaStreamDestroy(se.first);
  }
  if (p->run_stream) cudaStreamDestroy(p->run_stream);
  if (p->ring_stream) cudaStreamDestroy(p->ring_stream);
  if (p->dev) cudaFree(p->dev);
  if (p->pinned) cudaFreeHost(p->pinned);
  if (p->mapped) cudaFreeHost(p->mapped);
  if (p->base) cudaFree(p->base);
  delete p;
}

}  // namespace

extern "C" {

const char* rasp_pool_last_error(void) { return g_pool_err.c_str(); }

int rasp_pool_create(const rasp_config* cfg, uint64_t arena_bytes, rasp_pool** out) {
  if (!cfg || !out) return pfail(RASP_EINVAL, "config or out is NULL");
  if (cfg->arena) return pfail(RASP_EINVAL, "the pool owns its arena: rasp_config.arena must be NULL");
  *out = nullptr;
  {
    // the pool's requests are checked against cfg (w, semantics, l, s, flags) at submit
    const uint32_t one = 1;
    uint64_t bytes = 0;
    const int rc = rasp_batch_bytes(cfg, 1, &one, &bytes);
    if (rc) return pfail(rc, std::string("config rejected: ") + rasp_last_error());
  }
  rasp_pool* p = new (std::nothrow) rasp_pool();
  if (!p) return pfail(RASP_ENOMEM, "host allocation failed");
  p->cfg = *cfg;
  p->cfg.stream = nullptr;
  p->var.masked = cfg->word_bits < 64;
  p->var.checked = cfg->semantics == RASP_CHECKED;
  p->var.classic = (cfg->flags & RASP_ISA_CLASSIC) != 0;
  p->epoch = cfg->epoch ? cfg->epoch : 128u;
  arena_bytes = (arena_bytes + kAlign - 1) & ~(kAlign - 1);
  const size_t dev_bytes = sizeof(ServeSlot) * kMaxSlots + 4ull * kMaxSlots + 8ull * kRingCap + 256 + 16;
  void* base = nullptr;
  void* dev = nullptr;
  if (inject_alloc_failure() || cudaMalloc(&base, arena_bytes) != cudaSuccess ||
      cudaMalloc(&dev, dev_bytes) != cudaSuccess) {
    cudaGetLastError();
    if (base) cudaFree(base);
    delete p;
    return pfail(RASP_ENOMEM, "cudaMalloc of the pool arena or its ring failed");
  }
  p->base = (char*)base;
  p->dev = (char*)dev;
  p->bytes = arena_bytes;
  p->free_blocks[0] = arena_bytes;
  p->d_slots = (ServeSlot*)p->dev;
  p->d_pending = (uint32_t*)(p->d_slots + kMaxSlots);
  p->d_ring = (uint64_t*)(p->dev + ((sizeof(ServeSlot) * kMaxSlots + 4ull * kMaxSlots + 15) & ~15ull));
  p->d_head = (unsigned long long*)(p->d_ring + kRingCap);
  p->d_credits = p->d_head + 1;
  p->d_state = p->d_head + 2;
  void* pin = nullptr;
  void* map = nullptr;
  if (cudaHostAlloc(&pin, sizeof(ServeSlot) * kMaxSlots + 4ull * kMaxSlots, cudaHostAllocDefault) != cudaSuccess ||
      cudaHostAlloc(&map, 4ull * (kMaxSlots + 4), cudaHostAllocMapped) != cudaSuccess) {
    cudaGetLastError();
    if (pin) cudaFreeHost(pin);
    p->pinned = nullptr;
    free_pool(p);
    return pfail(RASP_ENOMEM, "cannot allocate the pool's host staging");
  }
  p->pinned = (char*)pin;
  p->mapped = (uint32_t*)map;
  memset(p->mapped, 0, 4ull * (kMaxSlots + 4));
  p->h_slots = (ServeSlot*)p->pinned;
  p->h_pending = (uint32_t*)(p->h_slots + kMaxSlots);
  void* dm = nullptr;
  if (cudaHostGetDevicePointer(&dm, map, 0) != cudaSuccess ||
      cudaStreamCreateWithFlags(&p->ring_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&p->run_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&p->published, cudaEventDisableTiming) != cudaSuccess ||
      cudaMemsetAsync(p->d_head, 0, 24, p->ring_stream) != cudaSuccess ||
      cudaStreamSynchronize(p->ring_stream) != cudaSuccess || serve_configure(p->var, p->shape) == 0) {
    cudaGetLastError();
    free_pool(p);
    return pfail(RASP_ECUDA, "cannot set up the serving ring");
  }
  p->d_mapped = (uint32_t*)dm;
  for (uint32_t k = kMaxSlots; k > 0; --k) p->free_slots.push_back(k - 1);
  *out = p;
  return RASP_OK;
}

int rasp_pool_submit(rasp_pool* p, const rasp_request* q, uint64_t* ticket) {
  if (!p || !q || !ticket) return pfail(RASP_EINVAL, "pool, request or ticket is NULL");
  if (!q->num_vms || !q->mem_words || !q->offsets || !q->tape_off)
    return pfail(RASP_EINVAL, "request needs num_vms, mem_words, offsets and tape_off");
  // a waiting request copies its inputs before they are validated by the
  // loads at admission: refuse buffers that the copy itself would read wrongly
  if (!q->num_programs) return pfail(RASP_EINVAL, "request has no programs");
  if (q->offsets[q->num_programs] && !q->words) return pfail(RASP_EINVAL, "words is NULL");
  if (q->tape_off[q->num_vms] && !q->tape) return pfail(RASP_EINVAL, "tape is NULL");
  if (q->num_vms > kRingCap) return pfail(RASP_ENOMEM, "request has more VMs than the serving ring holds");
  uint64_t need = 0;
  int rc = rasp_batch_bytes(&p->cfg, q->num_vms, q->mem_words, &need);
  if (rc) return pfail(rc, std::string("request rejected: ") + rasp_last_error());
  need = (need + kAlign - 1) & ~(kAlign - 1);
  if (need > p->bytes) return pfail(RASP_ENOMEM, "request needs more device memory than the whole pool");
  std::lock_guard<std::mutex> lock(p->mu);
  const uint64_t t = p->next_ticket++;
  Request& r = p->reqs[t];
  r.ticket = t;
  r.bytes = need;
  r.num_vms = q->num_vms;
  r.num_programs = q->num_programs;
  r.max_steps = q->max_steps;
  *ticket = t;
  uint64_t off = 0;
  if (p->waiting.empty() && reserve(p, q->num_vms, need, &off)) {
    // room now: load straight from the caller's buffers, no host copy
    r.offset = off;
    start(p, r, *q);
    if (r.state == RASP_REQ_DONE) p->done.push_back(t);             // failed at admission
    return RASP_OK;
  }
  const uint64_t nwords = q->offsets[q->num_programs];
  r.words.assign(q->words, q->words + nwords);
  r.offsets.assign(q->offsets, q->offsets + q->num_programs + 1);
  if (q->prog_of_vm) r.prog_of_vm.assign(q->prog_of_vm, q->prog_of_vm + q->num_vms);
  const uint64_t ntape = q->tape_off[q->num_vms];
  r.tape.assign(q->tape, q->tape + ntape);
  if (r.tape.empty()) r.tape.push_back(0);
  if (r.words.empty()) r.words.push_back(0);
  r.tape_off.assign(q->tape_off, q->tape_off + q->num_vms + 1);
  r.has_caps = q->caps != nullptr;
  if (q->caps) r.caps.assign(q->caps, q->caps + q->num_vms);
  r.mem_words.assign(q->mem_words, q->mem_words + q->num_vms);
  p->waiting.push_back(t);
  admit(p);
  *ticket = t;
  return RASP_OK;
}

int rasp_pool_poll(rasp_pool* p, uint64_t ticket, int* state) {
  if (!p || !state) return pfail(RASP_EINVAL, "pool or state is NULL");
  std::lock_guard<std::mutex> lock(p->mu);
  auto it = p->reqs.find(ticket);
  if (it == p->reqs.end()) return pfail(RASP_EINVAL, "unknown ticket");
  Request& r = it->second;
  if (check_done(p, r)) p->done.push_back(ticket);
  admit(p);
  *state = r.state;
  return RASP_OK;
}

int rasp_pool_next_done(rasp_pool* p, uint64_t* ticket) {
  if (!p || !ticket) return pfail(RASP_EINVAL, "pool or ticket is NULL");
  std::lock_guard<std::mutex> lock(p->mu);
  if (p->done.empty()) {
    // one pass over the running requests' completion words (in ticket order)
    for (auto& kv : p->reqs)
      if (check_done(p, kv.second)) p->done.push_back(kv.first);
    admit(p);
  }
  while (!p->done.empty()) {
    const uint64_t t = p->done.front();
    p->done.pop_front();
    if (p->reqs.count(t)) {        // still unread
      *ticket = t;
      return RASP_OK;
    }
  }
  *ticket = 0;
  return RASP_OK;
}

int rasp_pool_read(rasp_pool* p, uint64_t ticket, rasp_state_view* out) {
  if (!p) return pfail(RASP_EINVAL, "pool is NULL");
  std::lock_guard<std::mutex> lock(p->mu);
  auto it = p->reqs.find(ticket);
  if (it == p->reqs.end()) return pfail(RASP_EINVAL, "unknown ticket");
  Request& r = it->second;
  if (r.state == RASP_REQ_QUEUED) return pfail(RASP_ESTATE, "request not admitted yet");
  int rc = r.error;
  std::string msg = r.error_msg;
  if (!rc && r.state == RASP_REQ_RUNNING) {
    rc = wait_done(p, r);
    if (rc) msg = "the serving kernels returned before the request finished";
  }
  if (!rc && r.on_ring) {
    rc = device_error(p);
    if (rc) msg = "the serving kernel reported an internal error (a ring entry outside the slot table)";
  }
  if (!rc && r.batch && out) {
    rc = rasp_read_state(r.batch, 0, r.num_vms, out);
    if (rc) msg = rasp_last_error();
  }
  const bool stuck = r.state == RASP_REQ_RUNNING;   // its VMs may still be on the ring: keep the slot
  if (!stuck) {
    retire(p, r);
    p->completed++;
    p->reqs.erase(it);
  }
  admit(p);
  if (rc) return pfail(rc, msg);
  return RASP_OK;
}

int rasp_pool_cancel(rasp_pool* p, uint64_t ticket) {
  if (!p) return pfail(RASP_EINVAL, "pool is NULL");
  std::lock_guard<std::mutex> lock(p->mu);
  auto it = p->reqs.find(ticket);
  if (it == p->reqs.end()) return pfail(RASP_EINVAL, "unknown ticket");
  if (it->second.state != RASP_REQ_QUEUED)
    return pfail(RASP_ESTATE, "request already admitted; read it with rasp_pool_read");
  for (auto w = p->waiting.begin(); w != p->waiting.end(); ++w)
    if (*w == ticket) {
      p->waiting.erase(w);
      break;
    }
  p->reqs.erase(it);
  admit(p);                     // the next waiting request may fit now
  return RASP_OK;
}

int rasp_pool_info(rasp_pool* p, uint64_t* in_use, uint64_t* waiting, uint64_t* running) {
  if (!p) return pfail(RASP_EINVAL, "pool is NULL");
  std::lock_guard<std::mutex> lock(p->mu);
  uint64_t run = 0;
  for (auto& kv : p->reqs) run += kv.second.state == RASP_REQ_RUNNING;
  if (in_use) *in_use = p->in_use;
  if (waiting) *waiting = p->waiting.size();
  if (running) *running = run;
  return RASP_OK;
}

int rasp_pool_stats(rasp_pool* p, rasp_pool_counters* out) {
  if (!p || !out) return pfail(RASP_EINVAL, "pool or stats is NULL");
  std::lock_guard<std::mutex> lock(p->mu);
  memset(out, 0, sizeof(*out));
  out->admitted = p->admitted;
  out->completed = p->completed;
  out->kernel_launches = p->launches;
  out->kernel_returns = p->shape.grid ? (uint64_t)*exited_word(p) / p->shape.grid : 0;
  out->ring_published = p->tail;
  out->vms_in_flight = p->ring_used;
  out->kernel_ctas = p->shape.grid;
  return RASP_OK;
}

void rasp_pool_destroy(rasp_pool* p) {
  if (!p) return;
  {
    std::lock_guard<std::mutex> lock(p->mu);
    for (auto& kv : p->reqs) {
      Request& r = kv.second;
      if (r.state == RASP_REQ_RUNNING) wait_done(p, r);    // its VMs leave the ring before its memory goes
      retire(p, r);
    }
    p->reqs.clear();
  }
  free_pool(p);
}

}  // extern "C"
