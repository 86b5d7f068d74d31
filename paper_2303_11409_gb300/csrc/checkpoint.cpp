// Checkpoint of an MPS handle: mps_save writes the charge rule, the charge tables, the
// Schmidt values and the site blocks of the current state to a file, mps_load rebuilds a
// handle from it.  The state is the right-canonical form the update keeps
// (B = Gamma lambda per site, lambda per bond; Sec. II), so a loaded handle
// continues an evolution exactly where the saved one stopped.
//
// File layout (little-endian, all integers int32 unless noted):
//   "U1MPSCK1"                                   8-byte magic
//   version (3), L, d, N, chi_max, precision     (N encoded for several U(1) charges)
//   rule (version 3 only): kind (0 U(1), 1 Z_n, 2 several U(1)); Z_n: n; several U(1):
//                        ncomp, radix[ncomp], phys_charges[d * ncomp]
//   per bond b = 0..L:  n, charge[n], dim[n], lambda[sum dim] (float64)
//   per site s = 0..L-1: n_blocks (int32), nnz (int64), block (l, m) pairs
//                        [2 n_blocks], data[2 nnz] (float64, interleaved complex)
//   cut[L + 1] (float64): per bond, the relative cut of its last update, which
//                        sets the next update's SVD deflation level (versions 2, 3)
//   age[L + 1] (version 3 only): per bond, the update calls on the handle since that cut
//                        was recorded (the deflation level depends on it)
//   "U1MPSEND"                                   8-byte trailer
// Version 1 files (without the cut record) load with no deflation history, version 2 files
// with every cut one call old; both hold U(1) handles.
// The block order is the library's (l ascending, then m ascending), which the
// loader checks against the order the bond tables imply.
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <memory>
#include <new>
#include <stdexcept>
#include <string>
#include <vector>

#include "mps_internal.h"

namespace {

const char kMagic[8] = {'U', '1', 'M', 'P', 'S', 'C', 'K', '1'};
const char kTrailer[8] = {'U', '1', 'M', 'P', 'S', 'E', 'N', 'D'};

struct File {
  FILE* f = nullptr;
  ~File() { if (f) std::fclose(f); }
};

template <class T>
bool put(FILE* f, const T* p, size_t n) { return n == 0 || std::fwrite(p, sizeof(T), n, f) == n; }
template <class T>
bool get(FILE* f, T* p, size_t n) { return n == 0 || std::fread(p, sizeof(T), n, f) == n; }

// Bytes left between the read position and the end of the file (0 on error).  Every count
// read from the file is checked against it before anything is sized by that count, so a
// damaged or hostile file cannot make the loader allocate more than the file could hold.
int64_t remaining(FILE* f) {
  const long pos = std::ftell(f);
  if (pos < 0 || std::fseek(f, 0, SEEK_END) != 0) return 0;
  const long end = std::ftell(f);
  if (end < 0 || std::fseek(f, pos, SEEK_SET) != 0) return 0;
  return (int64_t)end - (int64_t)pos;
}

constexpr int64_t kMaxSites = int64_t(1) << 24;   // far above any chain a handle can hold
constexpr int32_t kAgeCap = 1 << 30;               // ages beyond this read as "long ago"
constexpr int64_t kCallBase = int64_t(1) << 40;    // call count of a loaded handle

// The charge rule of a version-3 file, read and checked before anything is created.
struct RuleRecord {
  int kind = 0, zn = 0, ncomp = 0;
  int32_t radix[4] = {};
  std::vector<int32_t> phys;   // d x ncomp
};

bool read_rule(FILE* f, int d, RuleRecord& r) {
  int32_t kind = -1;
  if (!get(f, &kind, 1)) return false;
  r.kind = kind;
  if (kind == 0) return true;
  if (kind == 1) {
    int32_t n = 0;
    if (!get(f, &n, 1) || n < d || n > mps::kMaxZn) return false;
    r.zn = n;
    return true;
  }
  if (kind != 2) return false;
  int32_t nc = 0;
  if (!get(f, &nc, 1) || nc < 1 || nc > 4) return false;
  r.ncomp = nc;
  if (!get(f, r.radix, nc)) return false;
  for (int k = 0; k < nc; ++k)
    if (r.radix[k] < 2) return false;
  r.phys.resize((size_t)d * nc);
  return get(f, r.phys.data(), r.phys.size());
}

int save_fail(mps_t h, const std::string& msg) {
  h->err = msg;
  return MPS_EINVAL;
}

}  // namespace

extern "C" {

int mps_save(mps_t h, const char* path) {
  if (!h) return MPS_EINVAL;
  if (!path) return save_fail(h, "path is NULL");
  for (int s = 0; s < h->L; ++s)
    if (h->dirty[s]) return save_fail(h, "site " + std::to_string(s) + " needs mps_set_site before saving");
  File out;
  out.f = std::fopen(path, "wb");
  if (!out.f) return save_fail(h, std::string("cannot open ") + path + " for writing");
  const int32_t hdr[6] = {3, h->L, h->d, h->N, h->chi_max, h->precision};
  bool ok = put(out.f, kMagic, 8) && put(out.f, hdr, 6);
  const mps::ChargeRule& R = h->rule;
  std::vector<int32_t> rule;
  if (R.multi) {
    rule = {2, R.ncomp};
    for (int k = 0; k < R.ncomp; ++k) rule.push_back(R.radix[k]);
    for (int i = 0; i < h->d; ++i) {   // decode q_i: first component most significant
      int64_t v = R.q[i];
      std::vector<int32_t> comp(R.ncomp);
      for (int k = R.ncomp - 1; k >= 0; --k) { comp[k] = (int32_t)(v % R.radix[k]); v /= R.radix[k]; }
      rule.insert(rule.end(), comp.begin(), comp.end());
    }
  } else if (R.zn) {
    rule = {1, R.zn};
  } else {
    rule = {0};
  }
  ok = ok && put(out.f, rule.data(), rule.size());
  std::vector<int32_t> ch, dm;
  std::vector<double> lam;
  for (int b = 0; ok && b <= h->L; ++b) {
    const mps::BondTable& t = h->bonds[b];
    const int n = t.size();
    ch.assign(t.charge.begin(), t.charge.end());
    dm.assign(t.dim.begin(), t.dim.end());
    lam.assign(t.total(), 0.0);
    int n_out = 0;
    int rc = mps_bond_spectrum(h, b, ch.data(), dm.data(), lam.data(), n, &n_out);
    if (rc != MPS_OK) return rc;
    ok = put(out.f, &n, 1) && put(out.f, ch.data(), n) && put(out.f, dm.data(), n) &&
         put(out.f, lam.data(), lam.size());
  }
  std::vector<int32_t> lc, mc, pairs;
  std::vector<double> data;
  for (int s = 0; ok && s < h->L; ++s) {
    const mps::SiteTable& S = h->sites[s];
    const int nb = (int)S.blocks.size();
    lc.resize(nb);
    mc.resize(nb);
    data.resize(2 * (size_t)S.nnz);
    int n_blocks = 0;
    int64_t n_values = 0;
    int rc = mps_get_site(h, s, lc.data(), mc.data(), nb, data.data(), S.nnz, &n_blocks, &n_values);
    if (rc != MPS_OK) return rc;
    pairs.resize(2 * (size_t)nb);
    for (int i = 0; i < nb; ++i) { pairs[2 * i] = lc[i]; pairs[2 * i + 1] = mc[i]; }
    const int64_t nnz = S.nnz;
    ok = put(out.f, &nb, 1) && put(out.f, &nnz, 1) && put(out.f, pairs.data(), pairs.size()) &&
         put(out.f, data.data(), data.size());
  }
  std::vector<double> cut(h->L + 1, 0.0);
  if ((int)h->cut_est.size() == h->L + 1) cut = h->cut_est;
  std::vector<int32_t> age(h->L + 1, kAgeCap);
  if ((int)h->cut_call.size() == h->L + 1)
    for (int b = 0; b <= h->L; ++b) age[b] = (int32_t)std::min<int64_t>(kAgeCap, h->calls - h->cut_call[b]);
  ok = ok && put(out.f, cut.data(), cut.size()) && put(out.f, age.data(), age.size()) && put(out.f, kTrailer, 8);
  if (!ok) return save_fail(h, std::string("write to ") + path + " failed");
  if (std::fclose(out.f) != 0) {
    out.f = nullptr;
    return save_fail(h, std::string("closing ") + path + " failed");
  }
  out.f = nullptr;
  return MPS_OK;
}

static int load_body(mps_t* out, const char* path, void* cuda_stream);

int mps_load(mps_t* out, const char* path, void* cuda_stream) {
  if (!out || !path) return MPS_EINVAL;
  *out = nullptr;
  // nothing may escape the C boundary: allocation failures and any other exception of the
  // host containers become status codes
  try {
    return load_body(out, path, cuda_stream);
  } catch (const std::bad_alloc&) {
    return MPS_ENOMEM;
  } catch (...) {
    return MPS_EINVAL;
  }
}

static int load_body(mps_t* out, const char* path, void* cuda_stream) {
  File in;
  in.f = std::fopen(path, "rb");
  if (!in.f) return MPS_EINVAL;
  char magic[8];
  int32_t hdr[6];
  if (!get(in.f, magic, 8) || std::memcmp(magic, kMagic, 8) != 0 || !get(in.f, hdr, 6) ||
      hdr[0] < 1 || hdr[0] > 3)
    return MPS_EINVAL;
  const int version = hdr[0];
  const int L = hdr[1], d = hdr[2], N = hdr[3], chi_max = hdr[4], precision = hdr[5];
  if (L < 2 || (int64_t)L > kMaxSites || d < 2 || d > MPS_MAX_D || N < 0 || chi_max < 1) return MPS_EINVAL;
  RuleRecord rule;
  if (version >= 3 && !read_rule(in.f, d, rule)) return MPS_EINVAL;
  // the total charge: a particle number (U(1)), a residue (Z_n) or an encoded vector
  if (rule.kind == 0 && (int64_t)N > (int64_t)L * (d - 1)) return MPS_EINVAL;
  if (rule.kind == 1 && (N >= rule.zn || (int64_t)N > (int64_t)L * (d - 1))) return MPS_EINVAL;
  // every bond record holds at least an int32 count, a charge, a dimension and one lambda
  if (remaining(in.f) < (int64_t)(L + 1) * 20) return MPS_EINVAL;
  // a product state of the same charge rule and total charge; every bond and site is then
  // overwritten (for several U(1) charges the left boundary charge is set afterwards)
  std::vector<int32_t> occ(L, 0);
  if (rule.kind != 2)
    for (int s = 0, left = N; s < L; ++s) { occ[s] = left < d - 1 ? left : d - 1; left -= occ[s]; }
  mps_t h = nullptr;
  int rc = MPS_OK;
  if (rule.kind == 0)
    rc = mps_create(&h, L, d, occ.data(), precision, chi_max, cuda_stream);
  else if (rule.kind == 1)
    rc = mps_create_cyclic(&h, L, d, rule.zn, occ.data(), precision, chi_max, cuda_stream);
  else
    rc = mps_create_multi(&h, L, d, rule.ncomp, rule.phys.data(), occ.data(), precision, chi_max, cuda_stream);
  if (rc != MPS_OK) return rc == MPS_ECHARGE ? MPS_EINVAL : rc;
  std::unique_ptr<mps_s, int (*)(mps_t)> guard(h, mps_destroy);
  if (rule.kind == 2) {
    for (int k = 0; k < rule.ncomp; ++k)
      if (h->rule.radix[k] != rule.radix[k]) return MPS_EINVAL;   // not the encoding of this rule
    h->bonds[0].charge[0] = N;
    h->N = N;
  }
  const int max_sectors = rule.kind == 0 ? N + 1 : chi_max;
  std::vector<int32_t> ch, dm;
  std::vector<double> lam;
  for (int b = 0; b <= L; ++b) {
    int32_t n = 0;
    if (!get(in.f, &n, 1) || n < 1 || n > max_sectors || (int64_t)n * 8 > remaining(in.f)) return MPS_EINVAL;
    ch.resize(n);
    dm.resize(n);
    if (!get(in.f, ch.data(), n) || !get(in.f, dm.data(), n)) return MPS_EINVAL;
    int64_t tot = 0;
    for (int i = 0; i < n; ++i) {
      if (dm[i] < 1 || dm[i] > chi_max) return MPS_EINVAL;
      tot += dm[i];
    }
    if (tot * 8 > remaining(in.f)) return MPS_EINVAL;
    lam.resize(tot);
    if (!get(in.f, lam.data(), tot)) return MPS_EINVAL;
    if (b == 0 || b == L) {   // boundary bonds: one sector (N at the left end, 0 at the right), lambda = 1
      if (n != 1 || dm[0] != 1 || ch[0] != (b == 0 ? N : 0) || lam[0] != 1.0) return MPS_ECHARGE;
      continue;
    }
    rc = mps_set_bond(h, b, n, ch.data(), dm.data(), lam.data());
    if (rc != MPS_OK) return rc;
  }
  std::vector<int32_t> pairs, lc, mc;
  std::vector<double> data;
  for (int s = 0; s < L; ++s) {
    int32_t nb = 0;
    int64_t nnz = 0;
    if (!get(in.f, &nb, 1) || !get(in.f, &nnz, 1) || nb < 0 || nnz < 0) return MPS_EINVAL;
    if (nnz > h->site_cap[s] || nb > (int64_t)h->site_cap[s]) return MPS_ENOMEM;
    if ((int64_t)nb * 8 + nnz * 16 > remaining(in.f)) return MPS_EINVAL;
    pairs.resize(2 * (size_t)nb);
    data.resize(2 * (size_t)nnz);
    if (!get(in.f, pairs.data(), pairs.size()) || !get(in.f, data.data(), data.size())) return MPS_EINVAL;
    lc.resize(nb);
    mc.resize(nb);
    for (int i = 0; i < nb; ++i) { lc[i] = pairs[2 * i]; mc[i] = pairs[2 * i + 1]; }
    mps::SiteTable t;
    mps::layout_site(h->bonds[s], h->bonds[s + 1], h->rule, t);
    if (t.nnz != nnz) return MPS_ECHARGE;   // the blocks do not fit the bond tables
    rc = mps_set_site(h, s, nb, lc.data(), mc.data(), data.data());
    if (rc != MPS_OK) return rc;
  }
  std::vector<double> cut(L + 1, 0.0);
  if (version >= 2) {
    if (!get(in.f, cut.data(), cut.size())) return MPS_EINVAL;
    for (double c : cut)
      if (!(c >= 0.0 && c <= 1.0)) return MPS_EINVAL;
  }
  std::vector<int32_t> age(L + 1, 0);   // older files: every cut recorded by the last call
  if (version >= 3) {
    if (!get(in.f, age.data(), age.size())) return MPS_EINVAL;
    for (int32_t a : age)
      if (a < 0 || a > kAgeCap) return MPS_EINVAL;
  }
  char trailer[8];
  if (!get(in.f, trailer, 8) || std::memcmp(trailer, kTrailer, 8) != 0) return MPS_EINVAL;
  h->cut_est = cut;   // after every mps_set_bond / mps_set_site, which clear it
  h->calls = kCallBase;
  h->cut_call.assign(L + 1, 0);
  for (int b = 0; b <= L; ++b) h->cut_call[b] = kCallBase - age[b];
  *out = guard.release();
  return MPS_OK;
}

}  // extern "C"
