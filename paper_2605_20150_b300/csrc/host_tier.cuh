// Host tier of the block records (Sec. 3.4).  Two forms:
//  - resident: every block record in pinned host memory (one array);
//  - tiered ("CPU tiered cache" over storage, Sec. 3.4): the records live in
//    an append-only log file -- the latest version of block k at index[k]
//    ("on re-admission, blocks are always fetched via Index[k]") -- and a
//    pool of P pinned record slots caches the blocks used recently (LRU).  A
//    load to the GPU copies from a pool slot, reading the record from the log
//    first on a miss; a write-back from the GPU lands in a pool slot, which
//    becomes dirty; a dirty slot is appended to the log when the pool
//    recycles it (dirty evictions go VRAM -> CPU -> storage, Sec. 3.4).
//    Compaction of the log is not part of this tier: superseded versions
//    stay in the file until the table is destroyed (the file is removed).
// Every GPU copy from or into a slot is followed by record_use(), so a slot
// is recycled only after the copies that use it have run.
#pragma once
#include <list>
#include <string>
#include <vector>

#include "common.cuh"

namespace tgs {

struct HostTier {
  bool tiered = false;
  uint64_t K = 0, rec_floats = 0;
  float* pinned = nullptr;  // resident: K records; tiered: P slots
  uint64_t P = 0;
  // tiered
  int fd = -1;
  std::string path;
  std::vector<uint64_t> index;  // K: byte offset of the latest record in the log
  uint64_t log_end = 0;
  std::vector<int64_t> slot_of;     // K
  std::vector<int64_t> block_of;    // P
  std::vector<uint8_t> dirty;       // P: newer than the log
  std::vector<cudaEvent_t> use_ev;  // P: the last GPU copy from or into the slot
  std::vector<uint8_t> use_pending;
  std::list<uint32_t> lru;  // slots, most recently used first
  std::vector<std::list<uint32_t>::iterator> lru_it;
  uint64_t hits = 0, misses = 0, bytes_read = 0, bytes_written = 0;

  // pool_blocks = 0 (or >= K): resident form; else tiered with a log file at
  // `file` (created, replaced, removed by release()).
  void init(uint64_t K, uint64_t rec_floats, uint64_t pool_blocks, const char* file);
  void release();
  uint64_t rec_bytes() const { return rec_floats * sizeof(float); }
  // Pinned record of block k for reading: the latest version (read from the
  // log into a slot on a miss).  Valid until the next acquire call.
  float* acquire_read(uint32_t k);
  // Pinned record of block k that a GPU write-back (or the host) will
  // overwrite: `whole` = the whole record is written (no read on a miss).
  // The slot becomes dirty.
  float* acquire_write(uint32_t k, bool whole);
  // After queueing a copy from / into block k's record on stream s.
  void record_use(uint32_t k, cudaStream_t s);
  // Writes a whole record of block k (set_params, resume).
  void put(uint32_t k, const float* rec);
  // Creation: block k's first record at log offset k x record size (several
  // threads may call it for different k); then finish_initial().
  void put_initial(uint32_t k, const float* rec);
  void finish_initial();
  // Invalidates the pool and restarts the log (set_params).
  void reset_log();

 private:
  uint32_t take_slot(uint32_t k);
  void touch(uint32_t slot);
  void write_back(uint32_t slot);
};

}  // namespace tgs
