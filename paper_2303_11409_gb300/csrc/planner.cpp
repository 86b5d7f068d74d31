// Integer sector planner of the two-site update (host side, bit-exact).
//
// arXiv:2303.11409, Sec. II: the Kronecker deltas of the U(1) amplitude formula
// allow a block (l, m) of a site only when c^[k-1] - c^[k] = i_k lies in
// [0, d-1]; a two-site update therefore couples the charges (l, m, r) of three
// consecutive bonds with 0 <= l-m <= d-1 and 0 <= m-r <= d-1, and its result
// splits by the new middle charge c into blocks Theta(c) whose rows are the left
// charges c <= l <= c+d-1 and whose columns are the right charges
// c-d+1 <= r <= c.  Because bond tables are sorted by charge, the rows and the
// columns of every Theta(c) are contiguous ranges of the left and right tables
// (the "charge-sorted memory alignment" of Sec. II).
#include <algorithm>
#include <new>
#include <cstring>

#include "mps_internal.h"

namespace mps {

int BondTable::find(int c) const {
  auto it = std::lower_bound(charge.begin(), charge.end(), c);
  if (it == charge.end() || *it != c) return -1;
  return (int)(it - charge.begin());
}

void BondTable::rebuild_offsets() {
  off.assign(charge.size() + 1, 0);
  for (size_t i = 0; i < charge.size(); ++i) off[i + 1] = off[i] + dim[i];
}

int SiteTable::find(int l, int m) const {
  // blocks are sorted by (l, m)
  int lo = 0, hi = (int)blocks.size();
  while (lo < hi) {
    int mid = (lo + hi) / 2;
    const SiteBlock& b = blocks[mid];
    if (b.l < l || (b.l == l && b.m < m)) lo = mid + 1; else hi = mid;
  }
  if (lo < (int)blocks.size() && blocks[lo].l == l && blocks[lo].m == m) return lo;
  return -1;
}

void layout_site(const BondTable& left, const BondTable& right, int d, SiteTable& out) {
  ChargeRule u1;
  u1.d = d;
  layout_site(left, right, u1, out);
}

void layout_site(const BondTable& left, const BondTable& right, const ChargeRule& rule, SiteTable& out) {
  out.blocks.clear();
  int64_t off = 0;
  for (int i = 0; i < left.size(); ++i) {
    for (int j = 0; j < right.size(); ++j) {
      if (rule.phys(left.charge[i], right.charge[j]) < 0) continue;
      SiteBlock b;
      b.l = left.charge[i]; b.m = right.charge[j];
      b.il = i; b.im = j;
      b.Dl = left.dim[i]; b.Dm = right.dim[j];
      b.off = off;
      off += (int64_t)b.Dl * b.Dm;
      out.blocks.push_back(b);
    }
  }
  out.nnz = off;
}

void plan_update(const BondTable& left, const BondTable& mid, const BondTable& right, int d,
                 UpdatePlan& plan) {
  ChargeRule u1;
  u1.d = d;
  plan_update(left, mid, right, u1, plan);
}

void ChargeRule::init_multi() {
  std::vector<int> tot;
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) tot.push_back(q[i] + q[j]);
  std::sort(tot.begin(), tot.end());
  tot.erase(std::unique(tot.begin(), tot.end()), tot.end());
  nb2 = (int)tot.size();
  int64_t off = 0;
  for (int k = 0; k < nb2; ++k) {
    q2[k] = tot[k];
    int n = 0;
    for (int i = 0; i < d; ++i) {
      pos2[k][i] = -1;
      for (int j = 0; j < d; ++j)
        if (q[i] + q[j] == tot[k]) { pos2[k][i] = (signed char)n++; break; }
    }
    sn2[k] = n;
    off2[k] = off;
    off += (int64_t)n * n;
  }
  off2[nb2] = off;
}

void ChargeRule::init_zn() {
  ztab = 1;
  nb2 = 0;
  int64_t off = 0;
  for (int t = 0; t < zn; ++t) {
    int n = 0;
    for (int i = 0; i < d; ++i) {
      pos2[nb2][i] = -1;
      if (wrap(t - i) < d) pos2[nb2][i] = (signed char)n++;
    }
    if (n == 0) continue;
    q2[nb2] = t;
    sn2[nb2] = n;
    off2[nb2] = off;
    off += (int64_t)n * n;
    ++nb2;
  }
  off2[nb2] = off;
}

static void fill_lists(const BondTable& left, const BondTable& right, SectorPlanEntry& e) {
  e.loff.clear();
  e.coff.clear();
  int o = 0;
  for (int i : e.li) { e.loff.push_back(o); o += left.dim[i]; }
  e.rows = o;
  o = 0;
  for (int j : e.ri) { e.coff.push_back(o); o += right.dim[j]; }
  e.cols = o;
  e.contiguous = true;
  for (size_t a = 1; a < e.li.size(); ++a) e.contiguous = e.contiguous && e.li[a] == e.li[a - 1] + 1;
}

void plan_update(const BondTable& left, const BondTable& mid, const BondTable& right, const ChargeRule& rule,
                 UpdatePlan& plan) {
  const int d = rule.d;
  plan.sectors.clear();
  plan.triple_l.clear(); plan.triple_m.clear(); plan.triple_r.clear();
  for (int i = 0; i < left.size(); ++i)
    for (int j = 0; j < mid.size(); ++j) {
      if (rule.phys(left.charge[i], mid.charge[j]) < 0) continue;
      for (int k = 0; k < right.size(); ++k) {
        if (rule.phys(mid.charge[j], right.charge[k]) < 0) continue;
        plan.triple_l.push_back(i); plan.triple_m.push_back(j); plan.triple_r.push_back(k);
      }
    }
  if (left.size() == 0 || right.size() == 0) return;
  if (rule.tabled()) {
    // several U(1) charges, or Z_n with d < n: every middle charge some (l, r) pair reaches,
    // with the left sectors l - c and the right sectors c - r among the physical charges (mod n
    // for Z_n) as rows and columns
    std::vector<int> cands;
    int buf[MPS_MAX_D];
    for (int i = 0; i < left.size(); ++i)
      for (int k = 0; k < right.size(); ++k) {
        const int n = rule.mids(left.charge[i], right.charge[k], buf);
        cands.insert(cands.end(), buf, buf + n);
      }
    std::sort(cands.begin(), cands.end());
    cands.erase(std::unique(cands.begin(), cands.end()), cands.end());
    for (int c : cands) {
      SectorPlanEntry e;
      e.c = c; e.l0 = e.l1 = e.r0 = e.r1 = -1;
      for (int i = 0; i < left.size(); ++i)
        if (rule.phys(left.charge[i], c) >= 0) e.li.push_back(i);
      for (int k = 0; k < right.size(); ++k)
        if (rule.phys(c, right.charge[k]) >= 0) e.ri.push_back(k);
      if (e.li.empty() || e.ri.empty()) continue;
      fill_lists(left, right, e);
      if (e.contiguous) { e.l0 = e.li.front(); e.l1 = e.li.back() + 1; }
      plan.sectors.push_back(e);
    }
    return;
  }
  if (rule.zn) {
    // Z_n with d = n: every middle charge c has all left sectors as rows (i' = (l - c) mod n)
    // and all right sectors as columns (j' = (c - r) mod n)
    for (int c = 0; c < rule.zn; ++c) {
      SectorPlanEntry e;
      e.c = c; e.l0 = 0; e.l1 = left.size(); e.r0 = 0; e.r1 = right.size();
      for (int i = e.l0; i < e.l1; ++i) e.li.push_back(i);
      for (int k = e.r0; k < e.r1; ++k) e.ri.push_back(k);
      fill_lists(left, right, e);
      plan.sectors.push_back(e);
    }
    return;
  }
  // Candidate middle charges: c with some left l in [c, c+d-1] and right r in [c-d+1, c].
  int cmin = std::max(right.charge.front(), left.charge.front() - (d - 1));
  int cmax = std::min(left.charge.back(), right.charge.back() + (d - 1));
  for (int c = cmin; c <= cmax; ++c) {
    // rows: left sectors with c <= l <= c + d - 1 (contiguous in the sorted table)
    int l0 = (int)(std::lower_bound(left.charge.begin(), left.charge.end(), c) - left.charge.begin());
    int l1 = (int)(std::upper_bound(left.charge.begin(), left.charge.end(), c + d - 1) - left.charge.begin());
    int r0 = (int)(std::lower_bound(right.charge.begin(), right.charge.end(), c - (d - 1)) - right.charge.begin());
    int r1 = (int)(std::upper_bound(right.charge.begin(), right.charge.end(), c) - right.charge.begin());
    if (l0 >= l1 || r0 >= r1) continue;
    SectorPlanEntry e;
    e.c = c; e.l0 = l0; e.l1 = l1; e.r0 = r0; e.r1 = r1;
    for (int i = l0; i < l1; ++i) e.li.push_back(i);
    for (int k = r0; k < r1; ++k) e.ri.push_back(k);
    fill_lists(left, right, e);
    plan.sectors.push_back(e);
  }
}

}  // namespace mps

using namespace mps;

static bool make_table(int n, const int32_t* c, const int32_t* dims, BondTable& t) {
  if (n < 0 || (n > 0 && (!c || !dims))) return false;
  t.charge.assign(c, c + n);
  t.dim.assign(dims, dims + n);
  for (int i = 0; i < n; ++i) {
    if (t.dim[i] < 1) return false;
    if (i && t.charge[i] <= t.charge[i - 1]) return false;
  }
  t.rebuild_offsets();
  return true;
}

static int plan_sectors_body(int d, int nl, const int32_t* lc, const int32_t* ld,
                                int nm, const int32_t* mc, const int32_t* md,
                                int nr, const int32_t* rc, const int32_t* rd,
                                int32_t* triples, int cap_triples, int* n_triples,
                                int32_t* sectors, int cap_sectors, int* n_sectors) {
  if (d < 2 || d > MPS_MAX_D || !n_triples || !n_sectors) return MPS_EINVAL;
  BondTable L, M, R;
  if (!make_table(nl, lc, ld, L) || !make_table(nm, mc, md, M) || !make_table(nr, rc, rd, R))
    return MPS_EINVAL;
  UpdatePlan p;
  plan_update(L, M, R, d, p);
  *n_triples = (int)p.triple_l.size();
  *n_sectors = (int)p.sectors.size();
  if (*n_triples > cap_triples || *n_sectors > cap_sectors) return MPS_EINVAL;
  if ((*n_triples && !triples) || (*n_sectors && !sectors)) return MPS_EINVAL;
  for (int t = 0; t < *n_triples; ++t) {
    triples[3 * t + 0] = L.charge[p.triple_l[t]];
    triples[3 * t + 1] = M.charge[p.triple_m[t]];
    triples[3 * t + 2] = R.charge[p.triple_r[t]];
  }
  for (int s = 0; s < *n_sectors; ++s) {
    sectors[3 * s + 0] = p.sectors[s].c;
    sectors[3 * s + 1] = p.sectors[s].rows;
    sectors[3 * s + 2] = p.sectors[s].cols;
  }
  return MPS_OK;
}

static int plan_sectors_rule_body(int d, int zn, int ncomp, const int32_t* phys_charges, const int32_t* radix,
                                     int nl, const int32_t* lc, const int32_t* ld,
                                     int nm, const int32_t* mc, const int32_t* md,
                                     int nr, const int32_t* rc, const int32_t* rd,
                                     int32_t* triples, int cap_triples, int* n_triples,
                                     int32_t* sectors, int cap_sectors, int* n_sectors,
                                     int32_t* lists, int cap_lists, int* n_lists) {
  if (d < 2 || d > MPS_MAX_D || !n_triples || !n_sectors || !n_lists) return MPS_EINVAL;
  if (zn < 0 || ncomp < 0 || ncomp > 4 || (zn && ncomp)) return MPS_EINVAL;
  if (zn && (zn < d || zn > kMaxZn)) return MPS_EINVAL;   // Z_n with d <= n
  ChargeRule rule;
  rule.d = d;
  rule.zn = zn;
  if (zn && d < zn) rule.init_zn();
  if (ncomp) {
    if (!phys_charges || !radix) return MPS_EINVAL;
    rule.multi = 1;
    rule.ncomp = ncomp;
    int64_t w = 1;
    int64_t weight[4];
    for (int k = ncomp - 1; k >= 0; --k) {
      if (radix[k] < 2) return MPS_EINVAL;
      rule.radix[k] = radix[k];
      weight[k] = w;
      w *= radix[k];
      if (w > (int64_t)1 << 30) return MPS_EINVAL;
    }
    for (int i = 0; i < d; ++i) {
      int64_t e = 0;
      for (int k = 0; k < ncomp; ++k) {
        const int v = phys_charges[i * ncomp + k];
        if (v < 0 || 2 * (int64_t)v >= radix[k]) return MPS_ECHARGE;
        e += v * weight[k];
      }
      rule.q[i] = (int)e;
      if (i && rule.q[i] <= rule.q[i - 1]) return MPS_ECHARGE;
    }
    rule.init_multi();
  }
  BondTable L, M, R;
  if (!make_table(nl, lc, ld, L) || !make_table(nm, mc, md, M) || !make_table(nr, rc, rd, R))
    return MPS_EINVAL;
  for (const BondTable* t : {&L, &M, &R})
    for (int c : t->charge) {
      if (zn && (c < 0 || c >= zn)) return MPS_ECHARGE;
      if (ncomp) {   // every component in [0, radix / 2): differences then decode uniquely
        int64_t v = c;
        for (int k = ncomp - 1; k >= 0; --k) {
          const int64_t x = v % rule.radix[k];
          if (v < 0 || 2 * x >= rule.radix[k]) return MPS_ECHARGE;
          v /= rule.radix[k];
        }
        if (v != 0) return MPS_ECHARGE;
      }
    }
  UpdatePlan p;
  plan_update(L, M, R, rule, p);
  int64_t nlist = 0;
  for (const SectorPlanEntry& e : p.sectors) nlist += (int64_t)e.li.size() + (int64_t)e.ri.size();
  *n_triples = (int)p.triple_l.size();
  *n_sectors = (int)p.sectors.size();
  *n_lists = (int)nlist;
  if (*n_triples > cap_triples || *n_sectors > cap_sectors || nlist > cap_lists) return MPS_EINVAL;
  if ((*n_triples && !triples) || (*n_sectors && !sectors) || (nlist && !lists)) return MPS_EINVAL;
  for (int t = 0; t < *n_triples; ++t) {
    triples[3 * t + 0] = L.charge[p.triple_l[t]];
    triples[3 * t + 1] = M.charge[p.triple_m[t]];
    triples[3 * t + 2] = R.charge[p.triple_r[t]];
  }
  int64_t o = 0;
  for (int s = 0; s < *n_sectors; ++s) {
    const SectorPlanEntry& e = p.sectors[s];
    sectors[5 * s + 0] = e.c;
    sectors[5 * s + 1] = e.rows;
    sectors[5 * s + 2] = e.cols;
    sectors[5 * s + 3] = (int)e.li.size();
    sectors[5 * s + 4] = (int)e.ri.size();
    for (int i : e.li) lists[o++] = L.charge[i];
    for (int k : e.ri) lists[o++] = R.charge[k];
  }
  return MPS_OK;
}

// The C entry points: no exception of the host containers crosses the C boundary.
extern "C" int mps_plan_sectors(int d, int nl, const int32_t* lc, const int32_t* ld,
                                int nm, const int32_t* mc, const int32_t* md,
                                int nr, const int32_t* rc, const int32_t* rd,
                                int32_t* triples, int cap_triples, int* n_triples,
                                int32_t* sectors, int cap_sectors, int* n_sectors) {
  try {
    return plan_sectors_body(d, nl, lc, ld, nm, mc, md, nr, rc, rd, triples, cap_triples, n_triples, sectors,
                             cap_sectors, n_sectors);
  } catch (const std::bad_alloc&) {
    return MPS_ENOMEM;
  } catch (...) {
    return MPS_EINVAL;
  }
}

extern "C" int mps_plan_sectors_rule(int d, int zn, int ncomp, const int32_t* phys_charges, const int32_t* radix,
                                     int nl, const int32_t* lc, const int32_t* ld,
                                     int nm, const int32_t* mc, const int32_t* md,
                                     int nr, const int32_t* rc, const int32_t* rd,
                                     int32_t* triples, int cap_triples, int* n_triples,
                                     int32_t* sectors, int cap_sectors, int* n_sectors,
                                     int32_t* lists, int cap_lists, int* n_lists) {
  try {
    return plan_sectors_rule_body(d, zn, ncomp, phys_charges, radix, nl, lc, ld, nm, mc, md, nr, rc, rd, triples,
                                  cap_triples, n_triples, sectors, cap_sectors, n_sectors, lists, cap_lists, n_lists);
  } catch (const std::bad_alloc&) {
    return MPS_ENOMEM;
  } catch (...) {
    return MPS_EINVAL;
  }
}

// Two-site gate layout of a charge rule: the block sizes in layout order and the flattened
// length (host code).  U(1): blocks n = 0..2(d-1) over (i, n - i); Z_n: the residues that some
// pair reaches; several U(1): the distinct vector totals q_i + q_j, lexicographic.
static int gate_layout_body(int d, int zn, int ncomp, const int32_t* phys_charges, int32_t* sizes, int cap,
                            int* n_blocks, int64_t* length) {
  if (d < 2 || d > MPS_MAX_D || zn < 0 || ncomp < 0 || ncomp > 4 || (zn && ncomp) || !n_blocks || !length)
    return MPS_EINVAL;
  if (zn && (zn < d || zn > kMaxZn)) return MPS_EINVAL;
  std::vector<int> sz;
  if (ncomp) {
    if (!phys_charges) return MPS_EINVAL;
    std::vector<std::vector<int64_t>> tot;
    for (int i = 0; i < d; ++i)
      for (int j = 0; j < d; ++j) {
        std::vector<int64_t> t(ncomp);
        for (int k = 0; k < ncomp; ++k) {
          const int32_t a = phys_charges[i * ncomp + k], b = phys_charges[j * ncomp + k];
          if (a < 0 || b < 0) return MPS_ECHARGE;
          t[k] = (int64_t)a + b;
        }
        tot.push_back(t);
      }
    std::sort(tot.begin(), tot.end());
    for (size_t a = 0; a < tot.size();) {
      size_t b = a;
      while (b < tot.size() && tot[b] == tot[a]) ++b;
      const int pairs = (int)(b - a);
      // pairs (i, j) with the same total; each i appears at most once when the charges are
      // distinct, so the block size is the pair count
      sz.push_back(pairs);
      a = b;
    }
    for (int i = 1; i < d; ++i)   // distinct charge vectors, ascending
      if (!std::lexicographical_compare(phys_charges + (i - 1) * ncomp, phys_charges + i * ncomp,
                                        phys_charges + i * ncomp, phys_charges + (i + 1) * ncomp))
        return MPS_ECHARGE;
  } else if (zn) {
    for (int t = 0; t < zn; ++t) {
      int n = 0;
      for (int i = 0; i < d; ++i) n += ((t - i) % zn + zn) % zn < d;
      if (n) sz.push_back(n);
    }
  } else {
    for (int n = 0; n <= 2 * (d - 1); ++n) sz.push_back(std::min(d - 1, n) - std::max(0, n - d + 1) + 1);
  }
  *n_blocks = (int)sz.size();
  int64_t len = 0;
  for (int v : sz) len += (int64_t)v * v;
  *length = len;
  if (sizes) {
    if (cap < *n_blocks) return MPS_EINVAL;
    for (int k = 0; k < *n_blocks; ++k) sizes[k] = sz[k];
  }
  return MPS_OK;
}

extern "C" int mps_gate_layout(int d, int zn, int ncomp, const int32_t* phys_charges, int32_t* sizes, int cap,
                               int* n_blocks, int64_t* length) {
  try {
    return gate_layout_body(d, zn, ncomp, phys_charges, sizes, cap, n_blocks, length);
  } catch (const std::bad_alloc&) {
    return MPS_ENOMEM;
  } catch (...) {
    return MPS_EINVAL;
  }
}
