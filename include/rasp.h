/*
 * rasp.h -- C ABI of the GB300 batched word-RASP engine (librasp_gb300.so).
 *
 * The engine advances many independent word-RASP machines
 *     c = <i, a, M, u, y>  in  C_w = W x W x W^n x W^(l+1) x W^(s+1)
 * ("Towards a Linear-Algebraic Hypervisor", Sec. 2.1) through the one-step
 * transition of Sec. 2.1 until each reaches a fixed point (F = {c : c -> c})
 * or its step cap -- the vectorised map Phi of Sec. 2 iterated on the GPU.
 *
 * Conventions shared by every call:
 *  - Return value: RASP_OK (0) or a negative rasp_err. Nothing throws across
 *    the ABI. rasp_last_error() returns a thread-local message describing the
 *    last failure on the calling thread.
 *  - Words are int64 two's complement; the machine treats them as w-bit
 *    vectors (Sec. 2.1, W = F_2^w), so "x mod n" uses the unsigned value.
 *  - Host pointers passed in are read before the call returns; the library
 *    keeps no reference to them. Device memory belongs to the batch, or is
 *    carved from the caller's arena (rasp_config.arena) which the caller owns
 *    and must keep alive until rasp_batch_destroy.
 *  - All device work of a batch is ordered on rasp_config.stream. rasp_run is
 *    asynchronous; rasp_read_state, rasp_read_stats and rasp_sync synchronise
 *    that stream.
 *  - VM outcomes (halt, timeout, fault) are status values, never errors.
 *  - Testing hook: with the environment variable RASP_FAULT_INJECT=alloc,
 *    every device allocation the library would make fails with RASP_ENOMEM
 *    (no CUDA call is made for it).
 */
#ifndef RASP_GB300_RASP_H
#define RASP_GB300_RASP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ------------------------------------------------------- */
enum rasp_err {
    RASP_OK = 0,
    RASP_EINVAL = -1,    /* bad argument (see each call)                     */
    RASP_ENOMEM = -2,    /* device memory (or the arena) too small            */
    RASP_ECUDA = -3,     /* a CUDA call failed; message in rasp_last_error    */
    RASP_ESTATE = -4,    /* call out of order (e.g. rasp_run before loads)    */
    RASP_EDEVICE = -5    /* a kernel reported an internal error (bounded wait
                            expired); the batch state is not trustworthy      */
};

/* ---- VM status (per machine) -------------------------------------------- */
enum rasp_status {
    RASP_RUNNING = 0,        /* neither halted nor out of steps              */
    RASP_HALTED = 1,         /* configuration is a fixed point (Sec. 2.1 F)  */
    RASP_TIMEOUT = 2,        /* steps == cap without reaching F              */
    RASP_FAULT_OVERFLOW = 3, /* CHECKED only: signed overflow in ADD or MUL  */
    RASP_FAULT_ADDR = 4      /* CHECKED only: fetch or operand out of [0, n) */
};

/* ---- semantics ---------------------------------------------------------- */
enum rasp_semantics {
    RASP_WRAP = 0,    /* the paper's machine: arithmetic mod 2^w, circular
                         memory (Sec. 2.1); never faults                      */
    RASP_CHECKED = 1  /* no counterpart in the paper: w must be 64; memory is
                         not circular and ADD/MUL are signed 64-bit. Per step,
                         in order: fetch needs 0 <= i < n-1 (else FAULT_ADDR);
                         a fixed point halts; ADD, MUL, STO, PRI and a firing
                         RD need 0 <= j < n (else FAULT_ADDR); ADD/MUL signed
                         overflow gives FAULT_OVERFLOW. A faulting step is not
                         applied and not counted.                           */
};

/* ---- flags -------------------------------------------------------------- */
#define RASP_SCHED_AUTO        0x00u  /* autotuned choice per memory bucket   */
#define RASP_SCHED_PLAIN       0x10u  /* one thread per VM, state in HBM      */
#define RASP_SCHED_PERSIST     0x20u  /* persistent workers, M staged in SMEM */
#define RASP_SCHED_PERSIST_GL  0x30u  /* persistent workers, M in HBM via L1  */
#define RASP_SCHED_SHARED      0x40u  /* one CTA per program, program words in
                                         SMEM, served from there to every VM
                                         that has not written into them; the
                                         c_0 pack then writes only the data
                                         words of each slab (a VM's first
                                         write into its program words copies
                                         the program into its slab), and the
                                         program words are filled in before
                                         M is read back or another schedule
                                         runs; needs prog_of_vm for sharing */
#define RASP_SCHED_MASK        0xF0u
#define RASP_DISPATCH_SELECT   0x000u /* branch-free guarded-sum step         */
#define RASP_DISPATCH_VOTE     0x100u /* warp opcode voting, one handler/group */
#define RASP_COLLECT_STATS     0x1000u /* count executed steps per opcode      */
#define RASP_SHARED_PROGRAM    0x2000u /* programs indexed by prog_of_vm       */
#define RASP_CUDA_GRAPH        0x4000u /* rasp_run replays a CUDA graph captured
                                          once per budget (cached, up to 8)   */
#define RASP_BUDGET_ROUNDS     0x10000u /* HBM-slab persistent schedule: always run
                                          in budget rounds (4096 x 8^k steps)
                                          with the still-running VMs compacted
                                          between rounds; by default only
                                          batches larger than the resident
                                          lanes do                             */
#define RASP_STEP_BLOCK        0x20000u /* HBM-slab persistent schedule: evaluate
                                          every step as one predicated block
                                          (the earlier form) instead of the
                                          epoch loop that leaves by warp vote;
                                          SMEM-staged and shared-program
                                          schedules: one step at a time per
                                          lane instead of the epoch loop      */
#define RASP_ISA_CLASSIC       0x8000u /* the classic RASP opcode set (Sec. 1.1)
                                          on the same words: opcode 3 is SUB
                                          (a - M_j mod 2^w), opcode 5 is BPA
                                          (jump when a > 0, a read as a w-bit
                                          two's complement integer). Plain and
                                          HBM-slab persistent schedules, select
                                          dispatch (EINVAL otherwise)          */

typedef struct rasp_config {
    uint32_t word_bits;  /* w, 2..64 (64 for RASP_CHECKED)                     */
    uint32_t semantics;  /* enum rasp_semantics                                */
    uint32_t in_cap;     /* l: input tape capacity (u holds l+1 words)         */
    uint32_t out_cap;    /* s: output capacity (y holds s+1 words)             */
    uint32_t flags;      /* RASP_SCHED_* | RASP_DISPATCH_* | RASP_COLLECT_STATS */
    uint32_t epoch;      /* steps between warp scheduling points; 0 = default  */
    uint32_t warps_per_cta; /* persistent kernels: warps per CTA (SMEM-staged
                            up to 8, HBM-slab up to 4); 0 = default           */
    uint32_t refill_min; /* persistent kernels: idle lanes that trigger a
                            refill (SMEM-staged), or stopped lanes that end
                            an epoch early (HBM-slab); 0 = default            */
    uint32_t ctas_per_sm;/* persistent kernels: resident CTAs per SM (fewer
                            resident VMs keep their memory in L1/L2);
                            0 = as many as fit                                */
    uint32_t reserved;   /* must be 0                                         */
    void*    stream;     /* cudaStream_t for all work of the batch; NULL = the
                            legacy default stream                              */
    void*    arena;      /* optional caller-owned device memory for the batch;
                            NULL = the library allocates with cudaMalloc       */
    uint64_t arena_bytes;/* size of arena (see rasp_batch_bytes)               */
} rasp_config;

typedef struct rasp_batch rasp_batch;   /* opaque */

/* Host-side view of machine state for reading and restoring.
 * Arrays are indexed by VM within the requested range [first, first+count).
 * Any pointer may be NULL to skip that field. */
typedef struct rasp_state_view {
    int64_t*  i;        /* [count] instruction counter (full w-bit word)      */
    int64_t*  a;        /* [count] accumulator                                */
    uint64_t* steps;    /* [count] applied transitions (= tau_h when halted)  */
    uint8_t*  status;   /* [count] enum rasp_status                           */
    uint32_t* uhead;    /* [count] u_0, the input read head                   */
    uint32_t* ylen;     /* [count] y_0, the output count                      */
    int64_t*  y;        /* [count * out_cap] y_1..y_s of each VM              */
    int64_t*  mem;      /* M of the VMs, concatenated in VM order (n_v words
                           each); NULL to skip                                */
    uint64_t  mem_words;/* capacity of mem in words (checked)                 */
} rasp_state_view;

typedef struct rasp_stats {
    uint64_t vm_steps;      /* sum of steps over all VMs                       */
    uint64_t running, halted, timeout, fault_overflow, fault_addr;
    uint64_t op_steps[8];   /* applied steps per opcode 1..7 (index 0 unused);
                               only with RASP_COLLECT_STATS                    */
    uint64_t pri_full;      /* PRI steps that found y full (same condition)   */
    uint64_t bnz_taken;     /* taken BNZ steps (same condition)               */
    uint64_t launches;      /* kernel launches of the last rasp_run            */
} rasp_stats;

/* Bytes of device memory a batch needs (for sizing rasp_config.arena).
 * Same argument rules as rasp_batch_create. */
int rasp_batch_bytes(const rasp_config* cfg, uint64_t num_vms,
                     const uint32_t* mem_words, uint64_t* out_bytes);

/* Create a batch of num_vms machines; mem_words[v] = n of VM v (>= 1).
 * Each machine lives in the configuration space of Sec. 2.1,
 * C_w = W x W x W^n x W^(l+1) x W^(s+1) (i, a, M, u, y), with its own n.
 * Allocates the structure-of-arrays state store (i, a, steps, cap, status,
 * u_0, y_0 per VM), the per-VM M slabs, the tapes and outputs, and buckets
 * the VMs by n for scheduling. No machine is runnable until both
 * rasp_load_programs and rasp_load_inputs have been called.
 * EINVAL: cfg NULL, w outside 2..64, CHECKED with w != 64, num_vms 0 or
 * >= 2^32, some n = 0 or n >= 2^31. ENOMEM: allocation or arena too small. */
int rasp_batch_create(const rasp_config* cfg, uint64_t num_vms,
                      const uint32_t* mem_words, rasp_batch** out);

/* Load programs and pack M = P 0^(n-2m) for every VM (c_0, Sec. 2.1).
 * words: flat program words; offsets[num_programs+1] delimit program p.
 * prog_of_vm: NULL (then num_programs must equal num_vms and VM v runs
 * program v) or [num_vms] program index per VM (one program shared by many
 * VMs, e.g. a rollout of one candidate over many inputs).
 * Resets i = a = 0, steps = 0, status = RUNNING, u_0 = y_0 = 0, y = 0.
 * EINVAL: odd program length, 2m > n of a VM using it, bad index. The copy
 * to the device is issued before the per-program checks run (so that they
 * overlap it); after a failed check the batch holds no programs and
 * rasp_reset / rasp_run return ESTATE until programs are loaded again. */
int rasp_load_programs(rasp_batch* b, const int64_t* words,
                       const uint64_t* offsets, uint64_t num_programs,
                       const uint32_t* prog_of_vm);

/* As rasp_load_programs, for programs whose words all lie in
 * [-2^31, 2^31): the words are given as int32 and stand for the same int64
 * values (sign extension), so half as many bytes cross to the device. When
 * the programs take at most half of mem_words words they stay on the device
 * as 4-byte words, and every pack (this call, rasp_reset) reads them there
 * and sign-extends them: half the program bytes per pack; the 8-byte copy is
 * made on the device only for the shared-program schedule and the read-back
 * of a lazily packed batch. Larger programs are copied into the batch's
 * machine memory (which c_0 overwrites) and widened on the device once the
 * checks have passed. Same arguments, errors and c_0 as rasp_load_programs;
 * after a failed check the batch holds no programs and its machine memory is
 * undefined until loaded again. */
int rasp_load_programs_i32(rasp_batch* b, const int32_t* words,
                           const uint64_t* offsets, uint64_t num_programs,
                           const uint32_t* prog_of_vm);

/* Load input tapes x (u = [0, x, 0^(l-|x|)], Sec. 2.1) and per-VM step
 * caps. tape/offsets[num_vms+1] as for programs; caps NULL = no cap
 * (UINT64_MAX). Resets u_0 = 0. EINVAL: |x| > l, offsets not increasing;
 * as for programs, after a failed check the batch holds no inputs until
 * they are loaded again. */
int rasp_load_inputs(rasp_batch* b, const int64_t* tape,
                     const uint64_t* offsets, const uint64_t* caps);

/* Re-pack c_0 for every VM from the programs and inputs already loaded
 * (device-side; no host copy). ESTATE if either is missing. */
int rasp_reset(rasp_batch* b);

/* Advance every RUNNING machine until it halts (fixed point), faults, or has
 * taken min(max_steps, cap_v) steps in total: the one-step transition of
 * Sec. 2.1 (the case equation over LOD, ADD, MUL, STO, BNZ, RD, PRI) applied
 * repeatedly, i.e. the vectorised map Phi of Sec. 2 iterated over the batch,
 * with halting on the fixed-point set F = {c : c -> c} of Sec. 2.1 and
 * resumable epochs as in the persistent workers of App. A (Alg. 1). steps is cumulative, so
 * rasp_run(T1) followed by rasp_run(T2) equals rasp_run(T2). A VM that stops
 * on the budget (max_steps < cap) stays RUNNING unless it is a fixed point.
 * Asynchronous on the batch stream. ESTATE before both loads. */
int rasp_run(rasp_batch* b, uint64_t max_steps);

/* Wait for the batch stream; EDEVICE if a kernel flagged an internal error. */
int rasp_sync(rasp_batch* b);

/* Copy state of VMs [first, first+count) into caller-owned host arrays
 * (synchronises the stream): each machine's configuration <i, a, M, u_0, y>
 * of Sec. 2.1 (u_0 the read head, y_0 the output count, y_1..y_s the
 * outputs), its applied steps (tau_h of Sec. 3 for a halted machine) and
 * status. EINVAL: range outside the batch, mem too small. */
int rasp_read_state(rasp_batch* b, uint64_t first, uint64_t count,
                    rasp_state_view* out);

/* Overwrite state of VMs [first, first+count) from host arrays (checkpoint
 * restore). NULL fields are left unchanged. EINVAL: u_0 > l, y_0 > s,
 * status outside the enum, mem too small. */
int rasp_load_state(rasp_batch* b, uint64_t first, uint64_t count,
                    const rasp_state_view* in);

/* Aggregate counters of the batch (synchronises the stream). */
int rasp_read_stats(rasp_batch* b, rasp_stats* out);

/* Halting-time histogram of the batch, computed on the device: the
 * distribution of tau_h (the number of steps after which a machine reached
 * its fixed point; "Towards a Linear-Algebraic Hypervisor", Sec. 3, Fig. 1b)
 * over the HALTED machines. edges[0..nbins] (host array, strictly
 * increasing) delimit the bins: counts[k] = number of HALTED VMs with
 * edges[k] <= steps < edges[k+1]. other (optional, 4 entries) receives the
 * number of RUNNING, TIMEOUT and faulted (either kind) VMs, and of HALTED
 * VMs outside [edges[0], edges[nbins]). counts and other are host arrays
 * owned by the caller. Synchronises the stream. EINVAL: nbins 0 or above
 * 4096, edges not strictly increasing. */
int rasp_halting_histogram(rasp_batch* b, const uint64_t* edges, uint32_t nbins,
                           uint64_t* counts, uint64_t* other);

/* The k HALTED machines with the largest tau_h, selected on the device --
 * the filter of a generate -> run -> filter search (busy beavers,
 * superoptimisation; "Towards a Linear-Algebraic Hypervisor", Sec. 3 and
 * Sec. 5). steps_out[k] and vm_out[k] (caller-owned host arrays) receive
 * tau_h and the VM index, best first; ties go to the smaller VM index, so
 * the result is unique. *found = number of entries written (fewer than k if
 * fewer VMs halted). Synchronises the stream. EINVAL: k = 0 or k > 1024. */
int rasp_top_halting(rasp_batch* b, uint32_t k, uint64_t* steps_out, uint32_t* vm_out,
                     uint32_t* found);

/* Measured schedule choice (the autotuner): times candidate schedules
 * (persistent over HBM slabs with several epochs and CTA shapes, plain, and
 * SMEM-staged where it fits, as its epoch loop and one step at a time) on
 * this batch from its current state with the
 * given step budget, `reps` times each, restoring the state after every
 * trial, then adopts the fastest for later rasp_run calls (replacing any
 * schedule flag of the config). The machine state is left unchanged.
 * Allocates a temporary snapshot of the state (ENOMEM if it does not fit).
 * Synchronises the stream. The trial times appear in rasp_describe.
 * With more than one memory-size bucket a second pass follows (coordinate
 * descent over the buckets): each bucket in turn tries the other schedules
 * and resident-CTA counts while the rest keep theirs, and keeps one only if
 * the whole run gets more than 1 % faster. Buckets whose choices differ run
 * as separate launches; the per-bucket trials appear in rasp_describe. */
int rasp_autotune(rasp_batch* b, uint64_t max_steps, uint32_t reps);

/* Pin the schedule of one memory-size bucket (its "index" in the "buckets"
 * list of rasp_describe: the size class, n <= 64, 128, 256, 512, 768, 1024,
 * 2048, 4096 and larger, counted from 0 whether or not it holds VMs):
 * sched is RASP_SCHED_PLAIN, _PERSIST or _PERSIST_GL (RASP_SCHED_AUTO
 * returns the bucket to the batch-wide setting); epoch, warps_per_cta and
 * ctas_per_sm as in rasp_config (0 = default). The launch plan is the
 * bucketing of Sec. 2.1 machines by n; results do not depend on it.
 * EINVAL: bucket out of range, a shared-program batch, or a schedule the
 * batch's opcode set does not run on. A later rasp_autotune replaces it. */
int rasp_plan_bucket(rasp_batch* b, uint32_t bucket, uint32_t sched, uint32_t epoch,
                     uint32_t warps_per_cta, uint32_t ctas_per_sm);

/* Describe the launch plan as JSON into buf (NUL-terminated): per memory
 * bucket its size class, VM count, schedule, grid, warps per CTA, resident
 * CTAs per SM, shared memory, epoch and refill threshold; the launches of a
 * run; the bytes of a word of M ("word_bytes": 4 for w <= 32 on the plain
 * and HBM-slab schedules, else 8) and of a program word as the pack reads it
 * ("program_word_bytes": 4 for programs kept as loaded by
 * rasp_load_programs_i32, else 8); whether runs replay a CUDA graph; the
 * autotuner's report. EINVAL if buf is too small. Does not touch the GPU. */
int rasp_describe(const rasp_batch* b, char* buf, uint64_t size);

/* ---- running a caller-owned state store without allocating ---------------
 * The paper has no counterpart to this call. It exists for callers that
 * cannot allocate at the moment they run machines: engines whose device
 * memory belongs to another framework's allocator (a cudaMalloc behind that
 * allocator's back breaks its accounting, and fails when it holds the free
 * memory), and real-time loops that must not allocate (cudaMalloc and
 * cudaFree can synchronise the device). rasp_run_static advances VMs
 * [0, num_vms) of a state store that the caller owns, in place, exactly as
 * rasp_run does (same statuses, same cumulative step budget), and calls no
 * cudaMalloc, cudaFree or other allocator.
 *
 * Its only extra memory is a fixed scratch area inside the library (a queue
 * of up to RASP_STATIC_MAX_VMS VM ids and a few counters, about 4 MiB) that
 * every GPU loading the library keeps until the process exits. The first
 * call on each device does a one-time set-up with that device current: it
 * looks up that area's device address and loads the call's kernels. Make
 * that first call before any stream capture. The set-up is cached per device
 * ordinal; after cudaDeviceReset on a device the cached address is stale, so
 * do not use this call on a device that was reset in the same process.
 * Every call on a device shares the area and resets its counters, so calls
 * whose work overlaps on the GPU (e.g. on two streams at once) race: order
 * them on one stream or serialise them.
 *
 * Layout of the caller's device buffers (all device pointers, the caller
 * owns them): i, a, steps, cap, status, uhead, ylen, n, mem_off are arrays
 * of num_vms entries as in rasp_state_view (cap = per-VM step cap). VM v's
 * memory is mem[mem_off[v] .. mem_off[v] + n[v]); mem holds mem_words
 * int64 words and is 16-byte aligned. For every VM, 1 <= n[v] <= 2^31-1,
 * mem_off[v] is even and mem_off[v] + n[v] rounded up to even is at most
 * mem_words. The tape of VM v (u_1..u_l, zero padded) is
 * tape[v*lp .. v*lp + l) and its output y_1..y_s is y[v*sp .. v*sp + s),
 * with lp, sp = in_cap, out_cap rounded up to even; tape and y 16-byte
 * aligned and num_vms*lp, num_vms*sp words long. Words must already be
 * reduced to w bits.
 * The per-VM layout is checked on the device: a RUNNING VM that breaks one
 * of the rules on n and mem_off is not run (its state is left unchanged)
 * and is counted in *rejected, an optional caller-owned device uint32 that
 * the call sets to 0 first (NULL: not reported).
 * Returns RASP_EINVAL for num_vms > RASP_STATIC_MAX_VMS, bad w/semantics,
 * NULL or misaligned buffers, mem_words = 0, RASP_ECUDA if a CUDA call
 * fails; the message goes to err_buf (if given). Asynchronous on `stream`. */
#define RASP_STATIC_MAX_VMS (1u << 20)

typedef struct rasp_static_run {
    int64_t*        i;
    int64_t*        a;
    uint64_t*       steps;
    const uint64_t* cap;
    uint8_t*        status;
    uint32_t*       uhead;
    uint32_t*       ylen;
    const uint32_t* n;
    const uint64_t* mem_off;
    int64_t*        mem;
    const int64_t*  tape;
    int64_t*        y;
    uint64_t        num_vms;
    uint32_t        word_bits;   /* w, 2..64 */
    uint32_t        semantics;   /* RASP_WRAP or RASP_CHECKED */
    uint32_t        in_cap;      /* l */
    uint32_t        out_cap;     /* s */
    uint64_t        max_steps;   /* cumulative budget, as for rasp_run */
    void*           stream;      /* cudaStream_t */
    char*           err_buf;     /* optional: receives an error message */
    uint32_t        err_buf_size;
    uint32_t        reserved;
    uint64_t        mem_words;   /* words in mem (bounds every VM's slab) */
    uint32_t*       rejected;    /* optional device word: VMs refused for their layout */
} rasp_static_run;

int rasp_run_static(const rasp_static_run* run);

/* ---- serving: continuous batching of rollout requests --------------------
 * (The paper evaluates fixed batches only; this is the request loop around
 * the same machine.) A pool owns one device arena of `arena_bytes`. Each
 * submitted request is a batch of its own (programs, tapes, caps, memory
 * sizes; all VMs of the pool share cfg's w, semantics, l, s and opcode set).
 * A request is admitted as soon as a first-fit block of the arena can hold
 * its batch (rasp_batch_bytes), one of the pool's 1024 request slots is free
 * and the pool's ring has room for its VMs (2^24 VMs admitted and unread at
 * most); otherwise it waits first-in-first-out. Admission loads the request
 * on its own stream and appends its VMs to a ring in device memory that all
 * admitted requests share; one persistent serving kernel drains that ring,
 * so the lanes that one request's finished VMs free are taken by the VMs of
 * whatever request comes next (continuous batching of lanes, not only of
 * memory). A request is DONE when its last VM has stopped (the kernel writes
 * a completion word in host-mapped memory; polling reads it without a CUDA
 * call). rasp_pool_read copies a finished request's state out and frees its
 * block and slot, which admits waiting requests. The serving kernel returns
 * by itself once the ring is empty (after a wait of about 3 ms, or at once
 * when a newer instance is queued); admission launches a new instance, so
 * nothing on the device waits on the host without a limit. The pool's calls
 * are serialised by an internal mutex; errors are reported by
 * rasp_pool_last_error (thread-local). cfg's schedule, dispatch and stats
 * flags do not apply to pools. */
typedef struct rasp_pool rasp_pool;

enum rasp_request_state { RASP_REQ_QUEUED = 0, RASP_REQ_RUNNING = 1, RASP_REQ_DONE = 2 };

typedef struct rasp_request {
    const int64_t*  words;        /* program words, as for rasp_load_programs      */
    const uint64_t* offsets;      /* [num_programs + 1]                            */
    uint64_t        num_programs;
    const uint32_t* prog_of_vm;   /* NULL or [num_vms]                             */
    const int64_t*  tape;         /* inputs, as for rasp_load_inputs               */
    const uint64_t* tape_off;     /* [num_vms + 1]                                 */
    const uint64_t* caps;         /* NULL or [num_vms]                             */
    const uint32_t* mem_words;    /* [num_vms]                                     */
    uint64_t        num_vms;
    uint64_t        max_steps;    /* budget of the request's single rasp_run       */
} rasp_request;

/* EINVAL if cfg->arena is set (the pool owns its arena); ENOMEM if the arena
 * cannot be allocated. */
int rasp_pool_create(const rasp_config* cfg, uint64_t arena_bytes, rasp_pool** out);
/* Copies the request's inputs (host memory), queues it and admits what fits.
 * EINVAL for a malformed request (no VMs or programs; mem_words, offsets or
 * tape_off NULL; words or tape NULL while the offsets ask for words), ENOMEM
 * if it could never fit the arena.
 * Load errors found at admission are reported by rasp_pool_read. */
int rasp_pool_submit(rasp_pool* p, const rasp_request* req, uint64_t* ticket);
/* Non-blocking: *state = enum rasp_request_state; also admits waiting work. */
int rasp_pool_poll(rasp_pool* p, uint64_t ticket, int* state);
/* Non-blocking: *ticket = a request that has finished (DONE, including one
 * that failed at admission or that rasp_pool_poll saw finish) and has not been
 * handed out by this call before nor read, or 0 if there is none now. One call
 * checks every running request, so a server need not poll its tickets one by
 * one. Also admits waiting work. */
int rasp_pool_next_done(rasp_pool* p, uint64_t* ticket);
/* Copy out a RUNNING or DONE request's final state (waits for it; out may be
 * NULL to discard), free its memory and forget the ticket. ESTATE while
 * still QUEUED. EDEVICE if every serving kernel has returned without
 * finishing the request, or the kernel flagged a ring entry outside the
 * slot table (the wait is bounded by the kernels, not by a clock). */
int rasp_pool_read(rasp_pool* p, uint64_t ticket, rasp_state_view* out);
/* Withdraw a request that is still waiting for admission (QUEUED): it is
 * forgotten and its ticket becomes unknown. ESTATE once it was admitted (read
 * it with rasp_pool_read instead), EINVAL for an unknown ticket. */
int rasp_pool_cancel(rasp_pool* p, uint64_t ticket);
/* Bytes of the arena in use, requests waiting, requests running. */
int rasp_pool_info(rasp_pool* p, uint64_t* in_use, uint64_t* waiting, uint64_t* running);

typedef struct rasp_pool_counters {
    uint64_t admitted;        /* requests put on the ring                     */
    uint64_t completed;       /* requests read back (or failed) and freed     */
    uint64_t kernel_launches; /* serving kernel instances launched            */
    uint64_t kernel_returns;  /* instances all of whose CTAs have returned    */
    uint64_t ring_published;  /* VMs ever put on the ring                     */
    uint64_t vms_in_flight;   /* VMs admitted and not yet read back           */
    uint64_t kernel_ctas;     /* CTAs per serving kernel instance             */
} rasp_pool_counters;

/* Counters of the pool (non-blocking). kernel_returns reaching
 * kernel_launches means no serving kernel is on the device. */
int rasp_pool_stats(rasp_pool* p, rasp_pool_counters* out);
/* Wait for the requests still running, discard every request (running,
 * done or waiting; their results are lost), free the arena and the pool.
 * NULL is a no-op. */
void rasp_pool_destroy(rasp_pool* p);
/* Thread-local description of the last pool error on this thread. */
const char* rasp_pool_last_error(void);

/* Free the batch (synchronises its stream first). NULL is a no-op. */
void rasp_batch_destroy(rasp_batch* b);

/* Thread-local description of the last error on this thread ("" if none). */
const char* rasp_last_error(void);

/* Library version string. */
const char* rasp_version(void);

#ifdef __cplusplus
}
#endif

#endif /* RASP_GB300_RASP_H */
