// pool.cu -- serving: continuous batching of rollout requests.
//
// A pool owns one device arena. A submitted request (programs, tapes, caps,
// memory sizes) is admitted as soon as a first-fit block of the arena can
// hold its batch; it then gets its own batch carved from that block and its
// own stream, is loaded and run, and completes independently of the others.
// Requests that do not fit wait first-in-first-out; reading a result frees
// its block and admits waiting requests. Admitted requests' kernels run
// concurrently on the device (their streams are independent), so work that
// arrives while other requests run overlaps with them.
#include <chrono>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/rasp.h"
#include "internal.h"

namespace {

thread_local std::string g_pool_err;

int pfail(int code, const std::string& msg) {
  g_pool_err = msg;
  return code;
}

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
  cudaEvent_t done = nullptr;
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
};

namespace {

constexpr uint64_t kAlign = 256;

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

void fail_request(Request& r, int code, const char* where) {
  r.state = RASP_REQ_DONE;
  r.error = code;
  r.error_msg = std::string(where) + ": " + rasp_last_error();
}

// Start one admitted request from the host inputs `q`: batch in its block,
// own stream, load, run.
void start(rasp_pool* p, Request& r, const rasp_request& q) {
  rasp_config c = p->cfg;
  c.arena = p->base + r.offset;
  c.arena_bytes = r.bytes;
  if (cudaStreamCreateWithFlags(&r.stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&r.done, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    r.state = RASP_REQ_DONE;
    r.error = RASP_ECUDA;
    r.error_msg = "cannot create a stream or event";
    return;
  }
  c.stream = r.stream;
  int rc = rasp_batch_create(&c, q.num_vms, q.mem_words, &r.batch);
  if (rc) return fail_request(r, rc, "create");
  rc = rasp_load_programs(r.batch, q.words, q.offsets, q.num_programs, q.prog_of_vm);
  if (rc) return fail_request(r, rc, "load_programs");
  rc = rasp_load_inputs(r.batch, q.tape, q.tape_off, q.caps);
  if (rc) return fail_request(r, rc, "load_inputs");
  rc = rasp_run(r.batch, q.max_steps);
  if (rc) return fail_request(r, rc, "run");
  cudaEventRecord(r.done, r.stream);
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

// Admit waiting requests in arrival order while the arena has room.
void admit(rasp_pool* p) {
  while (!p->waiting.empty()) {
    Request& r = p->reqs[p->waiting.front()];
    uint64_t off = 0;
    if (!carve(p, r.bytes, &off)) break;
    r.offset = off;
    p->waiting.pop_front();
    start(p, r, held_inputs(r));
    if (r.state == RASP_REQ_DONE) p->done.push_back(r.ticket);   // failed at admission
  }
}

}  // namespace

extern "C" {

const char* rasp_pool_last_error(void) { return g_pool_err.c_str(); }

int rasp_pool_create(const rasp_config* cfg, uint64_t arena_bytes, rasp_pool** out) {
  if (!cfg || !out) return pfail(RASP_EINVAL, "config or out is NULL");
  if (cfg->arena) return pfail(RASP_EINVAL, "the pool owns its arena: rasp_config.arena must be NULL");
  *out = nullptr;
  rasp_pool* p = new (std::nothrow) rasp_pool();
  if (!p) return pfail(RASP_ENOMEM, "host allocation failed");
  p->cfg = *cfg;
  p->cfg.stream = nullptr;
  arena_bytes = (arena_bytes + kAlign - 1) & ~(kAlign - 1);
  void* base = nullptr;
  if (rasp::inject_alloc_failure() || cudaMalloc(&base, arena_bytes) != cudaSuccess) {
    cudaGetLastError();
    delete p;
    return pfail(RASP_ENOMEM, "cudaMalloc of the pool arena failed");
  }
  p->base = (char*)base;
  p->bytes = arena_bytes;
  p->free_blocks[0] = arena_bytes;
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
  if (p->waiting.empty() && carve(p, need, &off)) {
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
  if (r.state == RASP_REQ_RUNNING) {
    const cudaError_t e = cudaEventQuery(r.done);
    if (e != cudaErrorNotReady) {
      r.state = RASP_REQ_DONE;
      if (e != cudaSuccess) {
        r.error = RASP_ECUDA;
        r.error_msg = cudaGetErrorString(e);
      }
      p->done.push_back(ticket);
    }
  }
  admit(p);
  *state = r.state;
  return RASP_OK;
}

int rasp_pool_next_done(rasp_pool* p, uint64_t* ticket) {
  if (!p || !ticket) return pfail(RASP_EINVAL, "pool or ticket is NULL");
  std::lock_guard<std::mutex> lock(p->mu);
  if (p->done.empty()) {
    // one pass over the running requests (in ticket order)
    for (auto& kv : p->reqs) {
      Request& r = kv.second;
      if (r.state != RASP_REQ_RUNNING) continue;
      const cudaError_t e = cudaEventQuery(r.done);
      if (e == cudaErrorNotReady) continue;
      r.state = RASP_REQ_DONE;
      if (e != cudaSuccess) {
        r.error = RASP_ECUDA;
        r.error_msg = cudaGetErrorString(e);
      }
      p->done.push_back(kv.first);
    }
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
  if (!rc && r.batch && out) {
    rc = rasp_read_state(r.batch, 0, r.num_vms, out);
    if (rc) msg = rasp_last_error();
  }
  if (r.batch) rasp_batch_destroy(r.batch);
  if (r.done) cudaEventDestroy(r.done);
  if (r.stream) cudaStreamDestroy(r.stream);
  if (r.state != RASP_REQ_QUEUED) release(p, r.offset, r.bytes);
  p->reqs.erase(it);
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

void rasp_pool_destroy(rasp_pool* p) {
  if (!p) return;
  {
    std::lock_guard<std::mutex> lock(p->mu);
    for (auto& kv : p->reqs) {
      Request& r = kv.second;
      if (r.batch) rasp_batch_destroy(r.batch);
      if (r.done) cudaEventDestroy(r.done);
      if (r.stream) cudaStreamDestroy(r.stream);
    }
    p->reqs.clear();
  }
  cudaFree(p->base);
  delete p;
}

}  // extern "C"
