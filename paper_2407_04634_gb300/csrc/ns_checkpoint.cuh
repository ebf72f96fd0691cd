// Checkpoint files of ns_solve.
//
// Layout: 8 bytes "NSCKPT01", the ns_checkpoint_info record, the solver state
// (host byte order; both hosts that build this library are little-endian), then
// a 64-bit checksum of every byte before it.  The checksum is FNV-1a (Fowler,
// Noll, Vo; offset basis 14695981039346656037, prime 1099511628211) taken over
// little-endian 64-bit words instead of bytes, a short tail zero-padded: eight
// times fewer multiplies than the byte form, for files of several GB.
//
// A writer goes to <path>.tmp and renames it over <path> only after the checksum
// was written and the file synced, so a process that dies mid-write leaves the
// previous checkpoint in place.  Device sections move through one pinned
// staging buffer, a chunk at a time.
#pragma once
#include <cuda_runtime.h>
#include <unistd.h>

#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <string>

#include "../../include/nullspace.h"

namespace ns {

constexpr char kCkptMagic[8] = {'N', 'S', 'C', 'K', 'P', 'T', '0', '1'};
constexpr int64_t kCkptVersion = 1;
constexpr size_t kCkptStage = size_t(8) << 20;

struct Fnv64 {
  uint64_t h = 14695981039346656037ull;
  unsigned char tail[8] = {};
  int nt = 0;
  void word(const unsigned char* b) {
    uint64_t w = 0;
    for (int i = 0; i < 8; ++i) w |= (uint64_t)b[i] << (8 * i);
    h = (h ^ w) * 1099511628211ull;
  }
  void add(const void* p, size_t len) {
    const unsigned char* b = static_cast<const unsigned char*>(p);
    while (len && nt) {
      tail[nt++] = *b++;
      --len;
      if (nt == 8) {
        word(tail);
        nt = 0;
      }
    }
    for (; len >= 8; b += 8, len -= 8) word(b);
    while (len) {
      tail[nt++] = *b++;
      --len;
    }
  }
  uint64_t value() const {
    Fnv64 c = *this;
    if (c.nt) {
      for (int i = c.nt; i < 8; ++i) c.tail[i] = 0;
      c.word(c.tail);
    }
    return c.h;
  }
};

class CkptWriter {
 public:
  CkptWriter() = default;
  CkptWriter(const CkptWriter&) = delete;
  CkptWriter& operator=(const CkptWriter&) = delete;
  ~CkptWriter() {
    if (f_) {
      fclose(f_);
      remove(tmp_.c_str());
    }
    if (stage_) cudaFreeHost(stage_);
  }
  bool open(const char* path) {
    if (!path || !*path) return false;
    path_ = path;
    tmp_ = path_ + ".tmp";
    f_ = fopen(tmp_.c_str(), "wb");
    ok_ = f_ != nullptr;
    put(kCkptMagic, sizeof kCkptMagic);
    return ok_;
  }
  void put(const void* p, size_t n) {
    if (!ok_ || !n) return;
    fnv_.add(p, n);
    ok_ = fwrite(p, 1, n, f_) == n;
  }
  // n device bytes at d; `s` is synchronized after each chunk
  cudaError_t put_device(const void* d, size_t n, cudaStream_t s) {
    cudaError_t e = stage();
    for (size_t off = 0; e == cudaSuccess && ok_ && off < n; off += kCkptStage) {
      const size_t c = std::min(kCkptStage, n - off);
      e = cudaMemcpyAsync(stage_, static_cast<const char*>(d) + off, c, cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e == cudaSuccess) put(stage_, c);
    }
    return e;
  }
  // checksum, sync, rename over the target; false if any write failed
  bool commit() {
    if (!f_) return false;
    const uint64_t c = fnv_.value();
    ok_ = ok_ && fwrite(&c, sizeof c, 1, f_) == 1 && fflush(f_) == 0 && fsync(fileno(f_)) == 0;
    ok_ = (fclose(f_) == 0) && ok_;
    f_ = nullptr;
    if (ok_) ok_ = rename(tmp_.c_str(), path_.c_str()) == 0;
    if (!ok_) remove(tmp_.c_str());
    return ok_;
  }

 private:
  cudaError_t stage() {
    if (stage_) return cudaSuccess;
    cudaError_t e = cudaMallocHost(&stage_, kCkptStage);
    if (e != cudaSuccess) stage_ = nullptr;
    return e;
  }
  FILE* f_ = nullptr;
  std::string path_, tmp_;
  Fnv64 fnv_;
  bool ok_ = false;
  void* stage_ = nullptr;
};

class CkptReader {
 public:
  CkptReader() = default;
  CkptReader(const CkptReader&) = delete;
  CkptReader& operator=(const CkptReader&) = delete;
  ~CkptReader() {
    if (f_) fclose(f_);
    if (stage_) cudaFreeHost(stage_);
  }
  // opens the file, checks its magic, version and length, reads the record
  ns_status open(const char* path, ns_checkpoint_info* info) {
    if (!path || !*path) return NS_ERR_IO;
    f_ = fopen(path, "rb");
    if (!f_) return NS_ERR_IO;
    if (fseek(f_, 0, SEEK_END) != 0) return NS_ERR_IO;
    const long sz = ftell(f_);
    if (sz < 0 || fseek(f_, 0, SEEK_SET) != 0) return NS_ERR_IO;
    size_ = (uint64_t)sz;
    ok_ = true;
    char magic[8];
    if (!get(magic, sizeof magic) || std::char_traits<char>::compare(magic, kCkptMagic, 8) != 0) return NS_ERR_IO;
    if (!get(info, sizeof *info) || info->version != kCkptVersion) return NS_ERR_IO;
    return NS_OK;
  }
  bool get(void* p, size_t n) {
    if (!ok_ || pos_ + n + sizeof(uint64_t) > size_) return ok_ = false;
    if (n && fread(p, 1, n, f_) != n) return ok_ = false;
    fnv_.add(p, n);
    pos_ += n;
    return true;
  }
  // n bytes into device memory at d; `s` is synchronized after each chunk
  cudaError_t get_device(void* d, size_t n, cudaStream_t s) {
    if (!stage_) {
      cudaError_t e = cudaMallocHost(&stage_, kCkptStage);
      if (e != cudaSuccess) {
        stage_ = nullptr;
        return e;
      }
    }
    for (size_t off = 0; ok_ && off < n; off += kCkptStage) {
      const size_t c = std::min(kCkptStage, n - off);
      if (!get(stage_, c)) break;
      cudaError_t e = cudaMemcpyAsync(static_cast<char*>(d) + off, stage_, c, cudaMemcpyHostToDevice, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  // the rest of the payload through the checksum (host only)
  bool skip_rest() {
    unsigned char buf[1 << 16];
    while (ok_ && pos_ + sizeof(uint64_t) < size_) {
      const size_t c = (size_t)std::min<uint64_t>(sizeof buf, size_ - sizeof(uint64_t) - pos_);
      if (!get(buf, c)) return false;
    }
    return ok_;
  }
  // true when everything was read, nothing is left and the checksum matches
  bool finish() {
    uint64_t c = 0;
    if (!ok_ || pos_ + sizeof c != size_ || fread(&c, sizeof c, 1, f_) != 1) return false;
    return c == fnv_.value();
  }
  bool ok() const { return ok_; }

 private:
  FILE* f_ = nullptr;
  uint64_t size_ = 0, pos_ = 0;
  Fnv64 fnv_;
  bool ok_ = false;
  void* stage_ = nullptr;
};

}  // namespace ns
