// Checkpoint of a handle on disk: gca_h2_save writes the cluster tree and
// the H^2 representation of Sect. 4 (ranks, pivots, block lists, V, E, S, N
// in float64), gca_h2_load reads it back and rebuilds the device handle
// through the import path, so that a program can skip the construction.
//
// File layout (little-endian, as written by this host):
//   char[8]  magic "GCAH2CK1"
//   Header   sizes and build parameters (below)
//   int32    perm[n], begin[nc], end[nc], child0[nc], child1[nc], level[nc]
//   int32    rank[nc], pivots[rank_sum], far[2 nfar], near[2 nnear]
//   float64  V[v_entries], E[e_entries], S[s_entries], N[n_entries]
//   uint64   FNV-1a hash of every byte before it
// The file is written next to its target and renamed into place, so a
// reader never sees a partial file under the target name.

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "internal.hpp"

namespace {

constexpr char kMagic[8] = {'G', 'C', 'A', 'H', '2', 'C', 'K', '1'};

struct Header {
  int32_t n, nc, nfar, nnear;
  int32_t op, k, m, reserved;
  int64_t rank_sum, v_entries, e_entries, s_entries, n_entries;
  int64_t n_singular[4];
  gca_params params;
};

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

int io_error(const std::string& msg) {
  gca::set_error(msg);
  return GCA_ERR_IO;
}

struct Writer {
  FILE* f = nullptr;
  Fnv fnv;
  bool ok = true;
  void put(const void* p, size_t n) {
    if (!ok || n == 0) return;
    fnv.add(p, n);
    ok = std::fwrite(p, 1, n, f) == n;
  }
};

struct Reader {
  FILE* f = nullptr;
  Fnv fnv;
  bool ok = true;
  void get(void* p, size_t n) {
    if (!ok || n == 0) return;
    ok = std::fread(p, 1, n, f) == n;
    if (ok) fnv.add(p, n);
  }
};

// one-sided nested representations only: the import path has no column side
// and no single-level blocks
bool saveable(int op) { return op == 0 || op == 5 || op == 6; }

}  // namespace

extern "C" int gca_h2_save(const gca_h2* h, const char* path) {
  if (!h || !path || !*path) {
    gca::set_error("gca_h2_save: NULL handle or empty path");
    return GCA_ERR_INVALID_ARG;
  }
  if (!saveable(h->op)) {
    gca::set_error("gca_h2_save: only the nested one-sided handles (single layer, nodal basis) are saved");
    return GCA_ERR_UNSUPPORTED;
  }
  Header hd{};
  hd.n = h->n;
  hd.nc = h->nc;
  hd.nfar = (int32_t)h->far_t.size();
  hd.nnear = (int32_t)h->near_t.size();
  hd.op = h->op;
  hd.k = h->k;
  hd.m = h->m;
  hd.rank_sum = h->rank_sum;
  hd.v_entries = h->v_entries;
  hd.e_entries = h->e_entries;
  hd.s_entries = h->s_entries;
  hd.n_entries = h->n_entries;
  for (int c = 0; c < 4; ++c) hd.n_singular[c] = h->n_singular[c];
  hd.params = h->params;
  try {
    std::vector<int32_t> rank(hd.nc), piv(hd.rank_sum), far(2 * (size_t)hd.nfar), near(2 * (size_t)hd.nnear);
    std::vector<double> V(hd.v_entries), E(hd.e_entries), S(hd.s_entries), N(hd.n_entries);
    gca_host_dump d{rank.data(), piv.data(), far.data(), near.data(), V.data(), E.data(), S.data(), N.data()};
    GCA_TRY(gca_h2_export(h, &d));
    const std::string tmp = std::string(path) + ".tmp";
    Writer w;
    w.f = std::fopen(tmp.c_str(), "wb");
    if (!w.f) return io_error("gca_h2_save: cannot open " + tmp + " for writing");
    w.put(kMagic, sizeof(kMagic));
    w.put(&hd, sizeof(hd));
    const std::vector<int>* tree[6] = {&h->perm, &h->begin, &h->end, &h->child0, &h->child1, &h->level};
    for (const auto* v : tree) w.put(v->data(), sizeof(int32_t) * v->size());
    w.put(rank.data(), sizeof(int32_t) * rank.size());
    w.put(piv.data(), sizeof(int32_t) * piv.size());
    w.put(far.data(), sizeof(int32_t) * far.size());
    w.put(near.data(), sizeof(int32_t) * near.size());
    for (const auto* v : {&V, &E, &S, &N}) w.put(v->data(), sizeof(double) * v->size());
    const uint64_t sum = w.fnv.h;
    if (w.ok) w.ok = std::fwrite(&sum, 1, sizeof(sum), w.f) == sizeof(sum);
    const bool closed = std::fclose(w.f) == 0;
    if (!w.ok || !closed) {
      std::remove(tmp.c_str());
      return io_error("gca_h2_save: writing " + tmp + " failed");
    }
    if (std::rename(tmp.c_str(), path) != 0) {
      std::remove(tmp.c_str());
      return io_error(std::string("gca_h2_save: cannot rename ") + tmp + " to " + path);
    }
  } catch (const std::bad_alloc&) {
    gca::set_error("gca_h2_save: host allocation failed");
    return GCA_ERR_OOM;
  }
  return GCA_OK;
}

extern "C" int gca_h2_load(const char* path, uint32_t flags, void* stream, gca_h2** out) {
  if (!out || !path || !*path) {
    gca::set_error("gca_h2_load: NULL output or empty path");
    return GCA_ERR_INVALID_ARG;
  }
  *out = nullptr;
  Reader r;
  r.f = std::fopen(path, "rb");
  if (!r.f) return io_error(std::string("gca_h2_load: cannot open ") + path);
  struct Closer {
    FILE* f;
    ~Closer() { std::fclose(f); }
  } closer{r.f};
  // the file's length bounds every count before anything is allocated
  if (std::fseek(r.f, 0, SEEK_END) != 0) return io_error(std::string("gca_h2_load: cannot seek in ") + path);
  const long flen = std::ftell(r.f);
  std::rewind(r.f);
  const std::string bad = std::string("gca_h2_load: ") + path + " is not a complete checkpoint";
  char magic[8];
  Header hd{};
  r.get(magic, sizeof(magic));
  r.get(&hd, sizeof(hd));
  if (!r.ok || std::memcmp(magic, kMagic, sizeof(kMagic)) != 0) return io_error(bad + " (header)");
  const int64_t len = flen;
  auto fits = [&](int64_t count, int64_t size) { return count >= 0 && count <= len / size; };
  if (hd.n < 1 || hd.nc < 1 || !fits(hd.n, 4) || !fits(hd.nc, 4) || !fits(hd.nfar, 8) || !fits(hd.nnear, 8) ||
      !fits(hd.rank_sum, 4) || !fits(hd.v_entries, 8) || !fits(hd.e_entries, 8) || !fits(hd.s_entries, 8) ||
      !fits(hd.n_entries, 8) || !saveable(hd.op))
    return io_error(bad + " (sizes)");
  const int64_t want = (int64_t)sizeof(kMagic) + (int64_t)sizeof(Header) +
                       4 * ((int64_t)hd.n + 6 * (int64_t)hd.nc + hd.rank_sum + 2 * (int64_t)hd.nfar +
                            2 * (int64_t)hd.nnear) +
                       8 * (hd.v_entries + hd.e_entries + hd.s_entries + hd.n_entries) + 8;
  if (want != len) return io_error(bad + " (length)");
  try {
    // arrays of at least one element, so that an empty one still has an
    // address (the import takes a null pointer for a missing array)
    auto ints = [](int64_t n) { return std::vector<int32_t>((size_t)std::max<int64_t>(n, 1)); };
    auto reals = [](int64_t n) { return std::vector<double>((size_t)std::max<int64_t>(n, 1)); };
    std::vector<int32_t> perm = ints(hd.n), begin = ints(hd.nc), end = ints(hd.nc), child0 = ints(hd.nc),
                         child1 = ints(hd.nc), level = ints(hd.nc), rank = ints(hd.nc), piv = ints(hd.rank_sum),
                         far = ints(2 * (int64_t)hd.nfar), near = ints(2 * (int64_t)hd.nnear);
    std::vector<double> V = reals(hd.v_entries), E = reals(hd.e_entries), S = reals(hd.s_entries),
                        N = reals(hd.n_entries);
    const int64_t int_counts[10] = {hd.n, hd.nc, hd.nc, hd.nc, hd.nc, hd.nc, hd.nc, hd.rank_sum,
                                    2 * (int64_t)hd.nfar, 2 * (int64_t)hd.nnear};
    std::vector<int32_t>* int_arrays[10] = {&perm, &begin, &end, &child0, &child1, &level, &rank, &piv, &far, &near};
    for (int a = 0; a < 10; ++a) r.get(int_arrays[a]->data(), sizeof(int32_t) * (size_t)int_counts[a]);
    const int64_t real_counts[4] = {hd.v_entries, hd.e_entries, hd.s_entries, hd.n_entries};
    std::vector<double>* real_arrays[4] = {&V, &E, &S, &N};
    for (int a = 0; a < 4; ++a) r.get(real_arrays[a]->data(), sizeof(double) * (size_t)real_counts[a]);
    const uint64_t sum = r.fnv.h;
    uint64_t stored = 0;
    if (r.ok) r.ok = std::fread(&stored, 1, sizeof(stored), r.f) == sizeof(stored);
    if (!r.ok) return io_error(bad + " (read)");
    if (stored != sum) return io_error(bad + " (checksum)");
    const gca_tree tree{hd.nc, perm.data(), begin.data(), end.data(), child0.data(), child1.data(), level.data()};
    const gca_host_dump d{rank.data(), piv.data(), far.data(), near.data(), V.data(), E.data(), S.data(), N.data()};
    GCA_TRY(gca_h2_import(&tree, hd.n, hd.nfar, hd.nnear, &d, flags, stream, out));
    // what the import cannot know: the construction's parameters and counts
    gca_h2* h = *out;
    h->k = hd.k;
    h->m = hd.m;
    for (int c = 0; c < 4; ++c) h->n_singular[c] = hd.n_singular[c];
    const uint32_t keep = h->params.flags;
    h->params = hd.params;
    h->params.flags = keep;
  } catch (const std::bad_alloc&) {
    if (*out) {
      gca_free(*out);
      *out = nullptr;
    }
    gca::set_error("gca_h2_load: host allocation failed");
    return GCA_ERR_OOM;
  }
  return GCA_OK;
}
