// Basis file: a checkpoint of a truncated basis F~ (Sec. "Subspace of the
// ground state"), so that a sampled basis is kept and reused instead of
// sampled again.  Host code only.
//
// Layout (little-endian, 40-byte header, then the words):
//   0..7    magic "MCDBASIS"
//   8..11   format version (1)
//   12..15  n_sites
//   16..19  N_up
//   20..23  N_dn
//   24..31  number of words N_f
//   32..39  FNV-1a 64-bit hash of the N_f words' bytes (Fowler, Noll, Vo)
//   40..    N_f uint64 words (up << n_sites | dn), strictly ascending
// Loading checks the magic, version, sector, size and hash, then installs the
// words through mcd_set_basis, which checks order and sector as for any basis.
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "mcd_internal.h"

namespace {

constexpr char kMagic[8] = {'M', 'C', 'D', 'B', 'A', 'S', 'I', 'S'};
constexpr uint32_t kVersion = 1;

struct FileHeader {
  char magic[8];
  uint32_t version, n_sites, n_up, n_dn;
  int64_t n;
  uint64_t hash;
};
static_assert(sizeof(FileHeader) == 40, "basis file header is 40 bytes");

// FNV-1a, 64-bit: offset basis 14695981039346656037, prime 2^40 + 2^8 + 0xb3
uint64_t fnv1a64(const void* p, size_t bytes) {
  const unsigned char* b = static_cast<const unsigned char*>(p);
  uint64_t h = 0xcbf29ce484222325ull;
  for (size_t i = 0; i < bytes; ++i) {
    h ^= b[i];
    h *= 0x100000001b3ull;
  }
  return h;
}

}  // namespace

extern "C" {

int mcd_save_basis(const mcd_ctx* cc, const char* path) {
  if (!cc || !path) return MCD_E_INVALID;
  mcd_ctx* c = const_cast<mcd_ctx*>(cc);
  if (!c->has_ham) return mcd::fail(c, MCD_E_STATE, "save_basis: no Hamiltonian (sector) set");
  int64_t n = 0;
  int st = mcd_get_basis(c, nullptr, 0, &n);
  if (st != MCD_OK) return st;
  if (n < 1) return mcd::fail(c, MCD_E_STATE, "save_basis: no basis");
  std::vector<uint64_t> w;
  try {
    w.resize(size_t(n));
  } catch (const std::bad_alloc&) {
    return mcd::fail(c, MCD_E_OOM, "save_basis: out of host memory");
  }
  st = mcd_get_basis(c, w.data(), n, &n);
  if (st != MCD_OK) return st;
  FileHeader h;
  std::memcpy(h.magic, kMagic, sizeof kMagic);
  h.version = kVersion;
  h.n_sites = uint32_t(c->n);
  h.n_up = uint32_t(c->n_up);
  h.n_dn = uint32_t(c->n_dn);
  h.n = n;
  h.hash = fnv1a64(w.data(), sizeof(uint64_t) * size_t(n));
  FILE* f = std::fopen(path, "wb");
  if (!f) return mcd::fail(c, MCD_E_INVALID, std::string("save_basis: cannot open ") + path);
  bool ok = std::fwrite(&h, sizeof h, 1, f) == 1 && std::fwrite(w.data(), sizeof(uint64_t), size_t(n), f) == size_t(n);
  ok = (std::fclose(f) == 0) && ok;
  return ok ? MCD_OK : mcd::fail(c, MCD_E_INVALID, std::string("save_basis: write failed: ") + path);
}

int mcd_load_basis(mcd_ctx* c, const char* path) {
  if (!c || !path) return MCD_E_INVALID;
  if (!c->has_ham) return mcd::fail(c, MCD_E_STATE, "load_basis: no Hamiltonian (sector) set");
  FILE* f = std::fopen(path, "rb");
  if (!f) return mcd::fail(c, MCD_E_INVALID, std::string("load_basis: cannot open ") + path);
  auto bad = [&](int status, const char* why) {
    std::fclose(f);
    return mcd::fail(c, status, std::string("load_basis: ") + why + ": " + path);
  };
  FileHeader h;
  if (std::fread(&h, sizeof h, 1, f) != 1) return bad(MCD_E_INVALID, "shorter than the header");
  if (std::memcmp(h.magic, kMagic, sizeof kMagic) != 0 || h.version != kVersion)
    return bad(MCD_E_INVALID, "not a basis file of this version");
  if (int(h.n_sites) != c->n || int(h.n_up) != c->n_up || int(h.n_dn) != c->n_dn)
    return bad(MCD_E_SECTOR, "sector (n_sites, N_up, N_dn) differs from the Hamiltonian's");
  if (std::fseek(f, 0, SEEK_END) != 0) return bad(MCD_E_INVALID, "cannot seek");
  const long size = std::ftell(f);
  if (h.n < 1 || h.n > 0x7FFFFFFF || size < 0 || int64_t(size) != int64_t(sizeof h) + 8 * h.n)
    return bad(MCD_E_INVALID, "word count does not match the file size");
  if (std::fseek(f, long(sizeof h), SEEK_SET) != 0) return bad(MCD_E_INVALID, "cannot seek");
  std::vector<uint64_t> w;
  try {
    w.resize(size_t(h.n));
  } catch (const std::bad_alloc&) {
    return bad(MCD_E_OOM, "out of host memory");
  }
  if (std::fread(w.data(), sizeof(uint64_t), size_t(h.n), f) != size_t(h.n)) return bad(MCD_E_INVALID, "short read");
  std::fclose(f);
  if (fnv1a64(w.data(), sizeof(uint64_t) * size_t(h.n)) != h.hash)
    return mcd::fail(c, MCD_E_INVALID, std::string("load_basis: hash mismatch: ") + path);
  return mcd_set_basis(c, w.data(), h.n);
}

}  // extern "C"
