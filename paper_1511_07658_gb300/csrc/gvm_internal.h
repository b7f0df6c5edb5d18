// Internal layouts shared by the host runtime and the device code of the
// GPU virtualization manager. Not part of the public ABI (see include/gvm.h).
#pragma once

#include <cuda.h>
#include <stdint.h>

namespace gvm {

// ---- tiling ---------------------------------------------------------------
constexpr int kThreads = 256;         // scheduler and task-kernel CTA size (8 warps)
constexpr int kFmaTile = 128;         // FMA SGEMM output tile (square)
constexpr int kFmaBK = 16;            // FMA SGEMM k-step
constexpr int kTcM = 128;             // tcgen05 tile rows (one TMEM lane per row)
constexpr int kTcN = 256;             // tcgen05 tile columns (fp32 TMEM columns)
constexpr int kTcBK = 32;             // bf16 k per pipeline stage (64-byte rows)
constexpr int kTcStages = 4;          // TMA -> MMA pipeline depth
constexpr int kSplitRows = 128;       // rows of A (or columns of B) per split tile
constexpr int64_t kVaddTileMin = 16384;
constexpr int64_t kVaddTileMax = 1 << 20;
constexpr int kProfSlots = 12;        // per-launch phase counters (see kProf*)

// Bytes of one pipeline stage: A hi, A lo (kTcM x kTcBK) and B^T hi, lo (kTcN x kTcBK).
constexpr uint32_t kTcStageBytes = (2u * kTcM + 2u * kTcN) * kTcBK * 2u;

// ---- task kinds, phases, flags ---------------------------------------------
enum : uint32_t { kTaskVadd = 1, kTaskSgemm = 2, kTaskVmul = 3 };
enum : uint32_t { kPhaseSplit = 0, kPhaseMain = 1 };
enum : uint32_t {
  kFlagNeedsReady = 1u,   // host-mode inputs: wait for the input stream's ready word
  kFlagNeedsD2H = 2u,     // host-mode output: the output stream copies and completes
  kFlagSplit3 = 4u,       // SGEMM on the split-bf16 tensor-core path
  kFlagDirectOut = 8u,    // host-mode output written by the kernel into host memory
  kFlagTmA = 16u,         // wide / TMA split3: tmA maps A (ingest copies it)
  kFlagTmB = 32u,         // TMA split3: tmB maps B in 32-row x 32-value boxes (ingest copies it)
  kFlagTmB3 = 64u,        // with kFlagTmB: tmB is 3D, one box lands a k-step's eight 32-column slabs
};

// Device status words (written to HostShared::status with the place in `where`).
enum : uint32_t {
  kStatusOk = 0,
  kStatusTimeout = 1,
  kStatusBadTask = 2,
};
enum : uint32_t {
  kWhereReadyWait = 1,
  kWhereSplitWait = 2,
  kWhereFullBarrier = 3,
  kWhereEmptyBarrier = 4,
  kWhereAccumBarrier = 5,
  kWhereQueueFull = 6,
  kWhereItemWait = 7,   // a warp waiting for its CTA's next claimed tile
  kWhereItemRing = 8,   // the claiming warp waiting for a free item slot
};

constexpr uint32_t kClaimLocked = 0x40000000u;  // claim counter while a slot is rewritten

// ---- task body: written by the host into its ring, copied by the device ----
// 384 bytes; the two tensor maps must stay 64-byte aligned (they are at 0, 128).
struct alignas(128) TaskBody {
  CUtensorMap tmA;  // kFlagTmA: binary32 A (m x k), box {kTcBK, 256} (wide) or {kTcBK, 128} (TMA form)
  CUtensorMap tmB;  // kFlagTmB: binary32 B (k x n), box {32, kTcBK}; kFlagTmB3: (32, k, n / 32), box {32, kTcBK, 8}
  uint32_t type;
  uint32_t flags;
  uint32_t rank;
  uint32_t slot;
  uint32_t tag;      // (seq + 1) truncated to 32 bits; never 0
  uint32_t ntiles;   // all tiles of the task (split + main)
  uint32_t nsplit;   // split tiles (split3 only)
  uint32_t tiles_m;
  uint32_t tiles_n;
  uint32_t kp;       // k rounded up to a multiple of 8 (split3 scratch row pitch)
  int32_t m;
  int32_t k;
  int64_t n;
  int64_t vadd_tile; // elements per vector-add tile
  uint64_t a, b, c;  // device addresses of the operands
  uint64_t scratch;  // device address of the split3 planes (A planes, then B^T planes)
  uint64_t scratch_b;// device address of the B^T planes
  uint64_t pad[3];
};
static_assert(sizeof(TaskBody) == 384, "TaskBody layout");

// Device task table entry: the body plus its counters on their own line.
struct alignas(128) DevTask {
  TaskBody body;
  uint32_t claimed[2];   // tiles claimed per phase
  uint32_t tiles_done;
  uint32_t split_done;
  uint64_t t_ingest;     // globaltimer when taken from the ring
  uint32_t pad2[26];
};
static_assert(sizeof(DevTask) == 512, "DevTask layout");

// Per-rank head word in pinned host memory, one per 64-byte line.
struct alignas(64) HostHead {
  uint32_t head;  // number of descriptors published by the host
  uint32_t pad[15];
};

// Completion record per ring slot in pinned host memory.
struct alignas(32) HostComplete {
  uint32_t tag;       // tag of the last completed task in this slot
  uint32_t pad;
  uint64_t t_ingest;  // device globaltimer, ns
  uint64_t t_done;
  uint64_t pad2;
};

// Host <-> device shared words (pinned host memory).
struct alignas(64) HostShared {
  uint32_t stop;        // host: scheduler should drain and exit
  uint32_t pad0[15];
  uint32_t exit_gen;    // device: launch generation of the last kernel that exited
  uint32_t pad1[15];
  uint32_t status;      // device: first error status
  uint32_t where;
  uint32_t info;
  uint32_t pad2[13];
  // device: timeline of the last scheduler launch that exited (globaltimer, ns)
  uint64_t k_start;      // first CTA started
  uint64_t k_last_done;  // last task completion
  uint64_t k_exit;       // last CTA left
  uint64_t k_prof[kProfSlots];  // per-phase CTA time summed over CTAs (kProf* order)
};

// Per-launch phase counters (nanoseconds of CTA time summed over CTAs, and counts).
enum : int {
  kProfAcquire = 0,    // the claiming warp finding the next tile (claims, ingest, idle polling)
  kProfIngest = 1,     // inside ingest passes that published work
  kProfStageWait = 2,  // split3: converters waiting for a free pipeline stage (MMA-bound time)
  kProfGemm = 3,       // GEMM tiles (FMA; split3: converter time, staging + epilogue)
  kProfMmaWait = 4,    // split3: the MMA warp waiting for a staged k-step (staging-bound time)
  kProfVadd = 5,       // vector-add tiles
  kProfTiles = 6,      // tiles run
  kProfIngests = 7,    // ingest passes that published work
  kProfEpilogue = 8,   // split3: converter time draining accumulators into C (part of kProfGemm)
};

// Device control block (front of the caller's ctrl buffer).
struct alignas(256) DevCtrl {
  uint32_t ingest_lock;
  uint32_t rr;            // next rank to start an ingest pass at
  uint32_t exit_count;
  uint32_t abort;
  uint64_t published;     // entries written to the publication queue
  uint64_t cursor;        // entries whose tiles have all been handed out (lower bound)
  uint32_t drained;       // drain mode: every published descriptor has been taken
  uint32_t pad0;
  uint64_t quiet_until;   // globaltimer before which look-ahead ingest is skipped
  uint64_t t_start;       // this launch: first CTA start (0 = unset)
  uint64_t t_last_done;   // this launch: last task completion
  uint64_t prof[kProfSlots];  // this launch: summed CTA time per phase (see kProf*)
  uint64_t published_tiles;  // tiles of all published entries (one global tile space)
  uint64_t next_tile;        // next tile index to hand out (may run ahead: a reservation)
  uint64_t first_entry;      // entries published before the current launch began
  uint32_t pad[18];
};
static_assert(sizeof(DevCtrl) == 256, "DevCtrl layout");

// Publication-queue entry: one phase of one task, covering tiles
// [base, base + cnt) of the global tile space.
struct PubEntry {
  uint64_t base;   // first global tile index
  uint64_t seq;    // entry index (checks that the ring slot was not reused)
  uint32_t task;   // rank * depth + slot
  uint32_t phase;  // kPhaseSplit or kPhaseMain
  uint32_t cnt;    // tiles in this entry
  uint32_t pad;
};
static_assert(sizeof(PubEntry) == 32, "PubEntry layout");

// Everything the scheduler kernel needs, passed by value.
struct SchedParams {
  DevCtrl* ctrl;
  uint32_t* tail;        // [ranks] descriptors consumed per rank
  uint32_t* ready;       // [ranks * depth] tag written by the input stream
  uint32_t* done;        // [ranks * depth] tag written by the scheduler (output stream waits)
  PubEntry* pubq;        // [qcap]
  DevTask* tasks;        // [ranks * depth]
  const TaskBody* host_desc;     // [ranks * depth] device view of the host ring
  const HostHead* host_heads;    // [ranks]
  HostComplete* host_complete;   // [ranks * depth]
  HostShared* host_shared;
  uint32_t ranks;
  uint32_t depth;        // power of two
  uint32_t qcap;         // power of two
  uint32_t quantum;
  uint32_t drain;        // 1: exit once every published descriptor is consumed
  uint32_t launch_gen;
  uint32_t prefetch;     // split3: prefetch the next queued tile's operands into L2
  uint32_t pad;
  uint64_t wait_timeout_ns;
  uint64_t idle_poll_ns;
};

// Control-block layout inside the caller's ctrl buffer.
struct CtrlLayout {
  uint64_t off_tail, off_ready, off_done, off_pubq, off_tasks, total;
  uint32_t qcap;
};

inline uint64_t align_up(uint64_t x, uint64_t a) { return (x + a - 1) / a * a; }

inline CtrlLayout ctrl_layout(uint32_t ranks, uint32_t depth) {
  CtrlLayout L;
  uint64_t slots = (uint64_t)ranks * depth;
  uint32_t q = 1;
  while (q < 4 * slots || q < 4096) q <<= 1;
  L.qcap = q;
  uint64_t off = sizeof(DevCtrl);
  L.off_tail = off;   off = align_up(off + 4ull * ranks, 256);
  L.off_ready = off;  off = align_up(off + 4ull * slots, 256);
  L.off_done = off;   off = align_up(off + 4ull * slots, 256);
  L.off_pubq = off;   off = align_up(off + sizeof(PubEntry) * (uint64_t)q, 256);
  L.off_tasks = off;  off = align_up(off + sizeof(DevTask) * slots, 256);
  L.total = off;
  return L;
}

// Split3 scratch: A planes [2][m][kp] then B^T planes [2][n][kp], bf16.
inline uint32_t split_kp(int32_t k) { return (uint32_t)((k + 7) / 8 * 8); }
inline uint64_t split_a_bytes(int32_t m, int32_t k) { return align_up(4ull * (uint64_t)m * split_kp(k), 256); }
inline uint64_t split_scratch_bytes(int32_t m, int32_t n, int32_t k) {
  return split_a_bytes(m, k) + align_up(4ull * (uint64_t)n * split_kp(k), 256);
}

}  // namespace gvm
