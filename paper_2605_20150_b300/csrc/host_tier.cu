// Host tier of the block records: pinned array, or a pinned LRU pool over an
// append-only log file (Sec. 3.4); see host_tier.cuh.
#include <fcntl.h>
#include <unistd.h>

#include <cerrno>
#include <cstring>

#include "host_tier.cuh"

namespace tgs {

namespace {

void full_pwrite(int fd, const void* buf, uint64_t bytes, uint64_t off) {
  const char* p = static_cast<const char*>(buf);
  while (bytes) {
    const ssize_t n = ::pwrite(fd, p, bytes > (1ull << 30) ? (1ull << 30) : bytes, (off_t)off);
    TGS_CHECK(n > 0, TGS_ERR_INVALID, std::string("host tier log write failed: ") + std::strerror(errno));
    p += n;
    off += (uint64_t)n;
    bytes -= (uint64_t)n;
  }
}

void full_pread(int fd, void* buf, uint64_t bytes, uint64_t off) {
  char* p = static_cast<char*>(buf);
  while (bytes) {
    const ssize_t n = ::pread(fd, p, bytes > (1ull << 30) ? (1ull << 30) : bytes, (off_t)off);
    TGS_CHECK(n > 0, TGS_ERR_INVALID, std::string("host tier log read failed: ") + std::strerror(errno));
    p += n;
    off += (uint64_t)n;
    bytes -= (uint64_t)n;
  }
}

}  // namespace

void HostTier::init(uint64_t k, uint64_t rf, uint64_t pool_blocks, const char* file) {
  K = k;
  rec_floats = rf;
  tiered = pool_blocks > 0 && pool_blocks < K;
  if (!tiered) {
    TGS_CUDA(cudaHostAlloc((void**)&pinned, K * rec_bytes(), cudaHostAllocPortable));
    return;
  }
  TGS_CHECK(file && file[0], TGS_ERR_INVALID, "a tiered host cache needs a backing file path");
  path = file;
  fd = ::open(file, O_RDWR | O_CREAT | O_TRUNC, 0600);
  TGS_CHECK(fd >= 0, TGS_ERR_INVALID, std::string("cannot open the host tier log: ") + file);
  P = pool_blocks;
  TGS_CUDA(cudaHostAlloc((void**)&pinned, P * rec_bytes(), cudaHostAllocPortable));
  index.assign(K, ~0ull);
  slot_of.assign(K, -1);
  block_of.assign(P, -1);
  dirty.assign(P, 0);
  use_ev.assign(P, nullptr);
  use_pending.assign(P, 0);
  lru_it.resize(P);
  lru.clear();
  for (uint64_t s = 0; s < P; ++s) {
    TGS_CUDA(cudaEventCreateWithFlags(&use_ev[s], cudaEventDisableTiming));
    lru.push_back((uint32_t)s);
    lru_it[s] = std::prev(lru.end());
  }
  log_end = 0;
}

void HostTier::release() {
  if (pinned) cudaFreeHost(pinned);
  pinned = nullptr;
  for (auto& e : use_ev)
    if (e) cudaEventDestroy(e);
  use_ev.clear();
  if (fd >= 0) {
    ::close(fd);
    ::unlink(path.c_str());
    fd = -1;
  }
}

void HostTier::reset_log() {
  if (!tiered) return;
  for (uint64_t s = 0; s < P; ++s) {
    if (use_pending[s]) TGS_CUDA(cudaEventSynchronize(use_ev[s]));
    use_pending[s] = 0;
    block_of[s] = -1;
    dirty[s] = 0;
  }
  slot_of.assign(K, -1);
  index.assign(K, ~0ull);
  log_end = 0;
  TGS_CHECK(::ftruncate(fd, 0) == 0, TGS_ERR_INVALID, "cannot truncate the host tier log");
}

void HostTier::touch(uint32_t slot) { lru.splice(lru.begin(), lru, lru_it[slot]); }

// Appends a dirty slot's record to the log (its copies have run).
void HostTier::write_back(uint32_t slot) {
  const int64_t b = block_of[slot];
  if (b < 0 || !dirty[slot]) return;
  full_pwrite(fd, pinned + (uint64_t)slot * rec_floats, rec_bytes(), log_end);
  index[b] = log_end;
  log_end += rec_bytes();
  bytes_written += rec_bytes();
  dirty[slot] = 0;
}

// The least recently used slot, freed for block k: its copies waited for,
// its record appended to the log if dirty.
uint32_t HostTier::take_slot(uint32_t k) {
  const uint32_t slot = lru.back();
  if (use_pending[slot]) {
    TGS_CUDA(cudaEventSynchronize(use_ev[slot]));
    use_pending[slot] = 0;
  }
  write_back(slot);
  if (block_of[slot] >= 0) slot_of[block_of[slot]] = -1;
  block_of[slot] = k;
  slot_of[k] = slot;
  touch(slot);
  return slot;
}

float* HostTier::acquire_read(uint32_t k) {
  if (!tiered) return pinned + (uint64_t)k * rec_floats;
  if (slot_of[k] >= 0) {
    ++hits;
    touch((uint32_t)slot_of[k]);
    return pinned + (uint64_t)slot_of[k] * rec_floats;
  }
  ++misses;
  const uint32_t slot = take_slot(k);
  float* rec = pinned + (uint64_t)slot * rec_floats;
  TGS_CHECK(index[k] != ~0ull, TGS_ERR_STATE, "host tier: block has no record in the log");
  full_pread(fd, rec, rec_bytes(), index[k]);
  bytes_read += rec_bytes();
  return rec;
}

float* HostTier::acquire_write(uint32_t k, bool whole) {
  if (!tiered) return pinned + (uint64_t)k * rec_floats;
  float* rec;
  if (slot_of[k] >= 0) {
    ++hits;
    const uint32_t slot = (uint32_t)slot_of[k];
    touch(slot);
    rec = pinned + (uint64_t)slot * rec_floats;
  } else {
    ++misses;
    const uint32_t slot = take_slot(k);
    rec = pinned + (uint64_t)slot * rec_floats;
    if (!whole && index[k] != ~0ull) {
      full_pread(fd, rec, rec_bytes(), index[k]);
      bytes_read += rec_bytes();
    }
  }
  dirty[slot_of[k]] = 1;
  return rec;
}

void HostTier::record_use(uint32_t k, cudaStream_t s) {
  if (!tiered) return;
  const int64_t slot = slot_of[k];
  if (slot < 0) return;
  TGS_CUDA(cudaEventRecord(use_ev[slot], s));
  use_pending[slot] = 1;
}

void HostTier::put(uint32_t k, const float* rec) {
  if (!tiered) {
    std::memcpy(pinned + (uint64_t)k * rec_floats, rec, rec_bytes());
    return;
  }
  if (slot_of[k] >= 0) {  // drop a cached copy (the log receives the new record)
    const uint32_t slot = (uint32_t)slot_of[k];
    if (use_pending[slot]) TGS_CUDA(cudaEventSynchronize(use_ev[slot]));
    use_pending[slot] = 0;
    dirty[slot] = 0;
    block_of[slot] = -1;
    slot_of[k] = -1;
    lru.splice(lru.end(), lru, lru_it[slot]);
  }
  full_pwrite(fd, rec, rec_bytes(), log_end);
  index[k] = log_end;
  log_end += rec_bytes();
  bytes_written += rec_bytes();
}

void HostTier::put_initial(uint32_t k, const float* rec) {
  if (!tiered) {
    std::memcpy(pinned + (uint64_t)k * rec_floats, rec, rec_bytes());
    return;
  }
  full_pwrite(fd, rec, rec_bytes(), (uint64_t)k * rec_bytes());
  index[k] = (uint64_t)k * rec_bytes();
}

void HostTier::finish_initial() {
  if (!tiered) return;
  log_end = K * rec_bytes();
  bytes_written += K * rec_bytes();
}

}  // namespace tgs
