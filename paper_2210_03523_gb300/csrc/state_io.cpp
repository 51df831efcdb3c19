// state_io.cpp -- checkpoint and resume of a solution: the element orders,
// the time and the ragged state in one host file, with a checksum so that a
// truncated or corrupted file is refused instead of loaded.  (The paper's
// runs restart from saved solutions, Sec. 3.3; the adaptation stages change
// the orders, so a checkpoint carries them.)
//
// File layout (little-endian, as on both x86-64 and Arm hosts):
//   8 bytes  magic "DGSTATE1"
//   int32    version (1)
//   int32    n_elem
//   int64    n_nodes
//   double   t
//   int32    orders[3 n_elem]
//   double   q[5 n_nodes]       (state layout of dg.h)
//   uint64   FNV-1a hash of every byte above after the magic
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <vector>

#include "dg_internal.h"

namespace {

constexpr char kMagic[8] = {'D', 'G', 'S', 'T', 'A', 'T', 'E', '1'};
constexpr int32_t kVersion = 1;

struct Fnv {
  uint64_t h = 1469598103934665603ull;
  void add(const void* p, size_t n) {
    const unsigned char* b = static_cast<const unsigned char*>(p);
    for (size_t i = 0; i < n; ++i) {
      h ^= b[i];
      h *= 1099511628211ull;
    }
  }
};

struct Header {
  int32_t version, n_elem;
  int64_t n_nodes;
  double t;
};

// reads and checks the header; on success the file is positioned at the orders
dg_status open_checked(const char* path, FILE** out, Header* h) {
  FILE* f = std::fopen(path, "rb");
  if (!f) return DG_ERR_ARG;
  char magic[8];
  if (std::fread(magic, 1, 8, f) != 8 || std::memcmp(magic, kMagic, 8) != 0 ||
      std::fread(&h->version, sizeof(int32_t), 1, f) != 1 || std::fread(&h->n_elem, sizeof(int32_t), 1, f) != 1 ||
      std::fread(&h->n_nodes, sizeof(int64_t), 1, f) != 1 || std::fread(&h->t, sizeof(double), 1, f) != 1 ||
      h->version != kVersion || h->n_elem <= 0 || h->n_nodes <= 0) {
    std::fclose(f);
    return DG_ERR_ARG;
  }
  *out = f;
  return DG_OK;
}

}  // namespace

extern "C" dg_status dg_state_write(const char* path, int32_t n_elem, const int32_t* orders, const double* q_host,
                                    double t) {
  if (!path || n_elem <= 0 || !orders || !q_host) return DG_ERR_ARG;
  int64_t n_nodes = 0;
  if (dg_count_nodes(n_elem, orders, &n_nodes) != DG_OK) return DG_ERR_ARG;
  FILE* f = std::fopen(path, "wb");
  if (!f) return DG_ERR_ARG;
  Fnv hash;
  bool ok = std::fwrite(kMagic, 1, 8, f) == 8;
  auto put = [&](const void* p, size_t sz, size_t n) {
    ok = ok && std::fwrite(p, sz, n, f) == n;
    hash.add(p, sz * n);
  };
  put(&kVersion, sizeof(int32_t), 1);
  put(&n_elem, sizeof(int32_t), 1);
  put(&n_nodes, sizeof(int64_t), 1);
  put(&t, sizeof(double), 1);
  put(orders, sizeof(int32_t), 3 * (size_t)n_elem);
  put(q_host, sizeof(double), 5 * (size_t)n_nodes);
  ok = ok && std::fwrite(&hash.h, sizeof(uint64_t), 1, f) == 1;
  ok = (std::fclose(f) == 0) && ok;
  return ok ? DG_OK : DG_ERR_ARG;
}

extern "C" dg_status dg_state_info(const char* path, int32_t* n_elem, int64_t* n_nodes, double* t) {
  if (!path) return DG_ERR_ARG;
  FILE* f = nullptr;
  Header h;
  dg_status st = open_checked(path, &f, &h);
  if (st != DG_OK) return st;
  std::fclose(f);
  if (n_elem) *n_elem = h.n_elem;
  if (n_nodes) *n_nodes = h.n_nodes;
  if (t) *t = h.t;
  return DG_OK;
}

extern "C" dg_status dg_state_read(const char* path, int32_t n_elem, int32_t* orders, double* q_host, double* t) {
  if (!path || n_elem <= 0 || !orders || !q_host) return DG_ERR_ARG;
  FILE* f = nullptr;
  Header h;
  dg_status st = open_checked(path, &f, &h);
  if (st != DG_OK) return st;
  if (h.n_elem != n_elem) {
    std::fclose(f);
    return DG_ERR_ARG;
  }
  std::vector<int32_t> o(3 * (size_t)n_elem);
  std::vector<double> q(5 * (size_t)h.n_nodes);
  uint64_t stored = 0;
  bool ok = std::fread(o.data(), sizeof(int32_t), o.size(), f) == o.size() &&
            std::fread(q.data(), sizeof(double), q.size(), f) == q.size() &&
            std::fread(&stored, sizeof(uint64_t), 1, f) == 1;
  char extra;
  ok = ok && std::fread(&extra, 1, 1, f) == 0;   // nothing after the hash
  std::fclose(f);
  if (!ok) return DG_ERR_ARG;
  int64_t nn = 0;
  if (dg_count_nodes(n_elem, o.data(), &nn) != DG_OK || nn != h.n_nodes) return DG_ERR_ARG;
  Fnv hash;
  hash.add(&h.version, sizeof(int32_t));
  hash.add(&h.n_elem, sizeof(int32_t));
  hash.add(&h.n_nodes, sizeof(int64_t));
  hash.add(&h.t, sizeof(double));
  hash.add(o.data(), sizeof(int32_t) * o.size());
  hash.add(q.data(), sizeof(double) * q.size());
  if (hash.h != stored) return DG_ERR_ARG;
  std::memcpy(orders, o.data(), sizeof(int32_t) * o.size());
  std::memcpy(q_host, q.data(), sizeof(double) * q.size());
  if (t) *t = h.t;
  return DG_OK;
}
