// Host-only driver of the checkpoint writer (test fixture): writes a record and a
// payload through ns::CkptWriter's host path, or abandons a write, so that the test
// can check the file against the documented format.  No device is touched.
//   ckpt_writer_host <path> commit <payload bytes>
//   ckpt_writer_host <path> abandon <payload bytes>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "../paper_2407_04634_gb300/csrc/ns_checkpoint.cuh"

int main(int argc, char** argv) {
  if (argc != 4) return 2;
  const bool commit = std::strcmp(argv[2], "commit") == 0;
  const size_t len = (size_t)std::strtoull(argv[3], nullptr, 10);
  ns_checkpoint_info c{};
  c.version = ns::kCkptVersion;
  c.m = 5;
  c.n = 4;
  c.d = 2;
  c.restart_len = 12;
  c.seed = 77;
  c.eps = 1e-3;
  c.k0 = 4;
  c.restarts = (int64_t)len;
  std::vector<unsigned char> payload(len);
  for (size_t i = 0; i < len; ++i) payload[i] = (unsigned char)(i * 37 + 11);
  ns::CkptWriter w;
  if (!w.open(argv[1])) return 3;
  w.put(&c, sizeof c);
  // in uneven pieces, so the word-wise checksum sees partial words
  size_t off = 0, piece = 1;
  while (off < len) {
    const size_t k = std::min(piece, len - off);
    w.put(payload.data() + off, k);
    off += k;
    piece = piece * 3 + 1;
  }
  if (!commit) return 0;  // the destructor abandons the write
  return w.commit() ? 0 : 4;
}
