// Internal declarations of the GB300 U(1) MPS library: handle state, host mirrors
// of the charge tables, and the descriptors the host planner hands to kernels.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <string>
#include <vector>

#include "mps_gb300.h"

namespace mps {

constexpr int kSvdSideStreams = 4;      // side streams for concurrent SVD kernel groups

// ---------------------------------------------------------------------------
// Charge arithmetic.  U(1) (zn = 0, Sec. II): block (l, m) of a site carries the physical
// index i = l - m and exists for 0 <= i <= d - 1; the two-site gate has blocks q = l - r in
// [0, 2(d-1)] over the pairs (i, q - i).  Z_n (zn = n >= d, the "more general Abelian" case
// of Sec. I): charges are residues mod n, i = (l - m) mod n must lie below d; for d = n every
// pair of charges occurs and gate block q in [0, n) acts on the n pairs (i, (q - i) mod n), and
// for d < n the gate blocks come from tables (ztab).  For U(1) and for Z_n with d = n a
// Theta(c) block's rows and columns are contiguous runs of the sorted bond tables (for Z_n:
// all sectors); for Z_n with d < n and for several U(1) charges (multi) they are listed.
// ---------------------------------------------------------------------------
constexpr int kMaxZn = 1 << 20;   // largest n of a Z_n handle (bond charges are residues)

struct ChargeRule {
  int d = 2;
  int zn = 0;
  // Several U(1) charges (multi = 1): physical index i carries the charge vector q_i, stored
  // encoded as one integer q[i] (mixed radix, first component most significant, ascending in
  // i); bond charges are encoded the same way.  The radix of every component exceeds twice
  // its largest bond value, so differences of charges decode uniquely and the integer order
  // of valid charges is their lexicographic order.  A Theta(c) block then has as rows the
  // left sectors l with l - c among the q[i] (not always a contiguous run of the bond table).
  // Two-site gate blocks are the distinct totals q[i] + q[j], ascending, each over its pairs
  // (i, j) with i ascending.
  int multi = 0;
  // Z_n with d < n (ztab = 1): physical index i = 0..d-1 carries charge i mod n; a block (l, m)
  // exists iff (l - m) mod n < d, and the two-site gate blocks are the residues q = (i + j) mod n
  // that some pair reaches, ascending, each over its pairs (i, (q - i) mod n), i ascending (the
  // tables below, filled by init_zn; for d = n every residue has all n pairs and no table is used)
  int ztab = 0;
  int q[MPS_MAX_D] = {};
  int ncomp = 1;
  int radix[4] = {1, 1, 1, 1};
  int nb2 = 0;
  int q2[MPS_MAX_D * MPS_MAX_D] = {};
  int sn2[MPS_MAX_D * MPS_MAX_D] = {};
  int64_t off2[MPS_MAX_D * MPS_MAX_D + 1] = {};
  signed char pos2[MPS_MAX_D * MPS_MAX_D][MPS_MAX_D] = {};
  void init_multi();                       // fills the two-site block tables from q[]
  void init_zn();                          // fills them for Z_n with d < n (sets ztab)
  bool tabled() const { return multi || ztab; }
  int wrap(int c) const { return zn ? ((c % zn) + zn) % zn : c; }
  int phys(int l, int m) const {           // physical index of block (l, m), or -1
    if (multi) {
      const int x = l - m;
      for (int i = 0; i < d; ++i)
        if (q[i] == x) return i;
      return -1;
    }
    const int i = zn ? wrap(l - m) : l - m;
    return (i >= 0 && i < d) ? i : -1;
  }
  int charge_of(int i) const { return multi ? q[i] : i; }   // (encoded) charge of physical index i
  int pair(int l, int r) const {           // two-site gate block of (l, r), or -1
    if (tabled()) {
      const int x = ztab ? wrap(l - r) : l - r;
      int lo = 0, hi = nb2 - 1;
      while (lo <= hi) {
        const int mid = (lo + hi) / 2;
        if (q2[mid] == x) return mid;
        if (q2[mid] < x) lo = mid + 1; else hi = mid - 1;
      }
      return -1;
    }
    if (zn) return wrap(l - r);
    const int q_ = l - r;
    return (q_ >= 0 && q_ <= 2 * (d - 1)) ? q_ : -1;
  }
  int nblocks() const { return tabled() ? nb2 : (zn ? zn : 2 * d - 1); }
  int base(int q_) const { return zn ? 0 : (q_ - d + 1 > 0 ? q_ - d + 1 : 0); }   // first left index of block q (U(1))
  int sn(int k) const {
    if (tabled()) return sn2[k];
    return zn ? zn : (k < d - 1 ? k : d - 1) - base(k) + 1;
  }
  int gpos(int k, int i) const { return tabled() ? pos2[k][i] : i - base(k); }   // row of left index i in block k
  int64_t block_off(int k) const {
    if (tabled()) return off2[k];
    int64_t t = 0;
    for (int j = 0; j < k; ++j) t += (int64_t)sn(j) * sn(j);
    return t;
  }
  int64_t gate_len() const { return block_off(nblocks()); }
  // candidate middle charges c of a pair (l, r): [cmin, cmax] (U(1), Z_n)
  int cmin(int l, int r) const { return zn ? 0 : (r > l - d + 1 ? r : l - d + 1); }
  int cmax(int l, int r) const { return zn ? zn - 1 : (l < r + d - 1 ? l : r + d - 1); }
  // the middle charges of a pair (l, r), ascending, into out[MPS_MAX_D]; returns their count
  int mids(int l, int r, int* out) const {
    int n = 0;
    if (multi) {
      for (int i = d - 1; i >= 0; --i)
        if (phys(l - q[i], r) >= 0) out[n++] = l - q[i];
      return n;
    }
    if (ztab) {   // c = (l - i) mod n for a physical i, with (c - r) mod n < d; ascending
      for (int i = 0; i < d; ++i) {
        const int c = wrap(l - i);
        if (phys(c, r) < 0) continue;
        int k = n++;
        for (; k > 0 && out[k - 1] > c; --k) out[k] = out[k - 1];
        out[k] = c;
      }
      return n;
    }
    for (int c = cmin(l, r); c <= cmax(l, r); ++c) out[n++] = c;
    return n;
  }
};

// ---------------------------------------------------------------------------
// Host mirror of the charge structure (Sec. II: right-charge labels per bond,
// blocks (l, m) with a physical index i = l - m (mod n for Z_n) in [0, d-1] per site).
// ---------------------------------------------------------------------------
struct BondTable {
  std::vector<int> charge;    // ascending
  std::vector<int> dim;       // sector dimensions
  std::vector<int> off;       // prefix sums of dim (size n+1): lambda offset of each sector
  int total() const { return off.empty() ? 0 : off.back(); }
  int size() const { return (int)charge.size(); }
  int find(int c) const;      // sector index of charge c, or -1
  void rebuild_offsets();
};

struct SiteBlock {
  int l, m;        // bond-s charge, bond-(s+1) charge
  int il, im;      // sector indices in the two bond tables
  int Dl, Dm;
  int64_t off;     // offset of the block in the site slot, complex numbers
};

struct SiteTable {
  std::vector<SiteBlock> blocks;   // (l ascending, m ascending)
  int64_t nnz = 0;
  int find(int l, int m) const;    // block index or -1
};

// Enumerate the allowed blocks of a site between two bond tables, in (l, m) order.
void layout_site(const BondTable& left, const BondTable& right, int d, SiteTable& out);
void layout_site(const BondTable& left, const BondTable& right, const ChargeRule& rule, SiteTable& out);

// ---------------------------------------------------------------------------
// Sector plan of one two-site update (the integer planner, K0).
// ---------------------------------------------------------------------------
struct SectorPlanEntry {
  int c;             // candidate middle charge
  int l0, l1;        // row sectors: indices [l0, l1) of the left bond table (U(1), Z_n)
  int r0, r1;        // column sectors: indices [r0, r1) of the right bond table (U(1), Z_n)
  int rows, cols;    // Theta(c) size
  // the row / column sectors in order with their offsets inside Theta(c) (every rule; for
  // U(1) and Z_n the runs above); contiguous == the rows are one run of the left table
  std::vector<int> li, loff, ri, coff;
  bool contiguous = true;
  int row_off(int i) const {        // offset of left sector i, or -1
    for (size_t a = 0; a < li.size(); ++a)
      if (li[a] == i) return loff[a];
    return -1;
  }
  int col_off(int j) const {
    for (size_t a = 0; a < ri.size(); ++a)
      if (ri[a] == j) return coff[a];
    return -1;
  }
};
struct UpdatePlan {
  std::vector<SectorPlanEntry> sectors;                 // c ascending
  std::vector<int> triple_l, triple_m, triple_r;        // sector indices, lexicographic
};
void plan_update(const BondTable& left, const BondTable& mid, const BondTable& right, int d,
                 UpdatePlan& plan);
void plan_update(const BondTable& left, const BondTable& mid, const BondTable& right, const ChargeRule& rule,
                 UpdatePlan& plan);

// ---------------------------------------------------------------------------
// Kernel descriptors (plain structs, copied to device memory in one upload).
// ---------------------------------------------------------------------------
struct ThetaTask {            // one (l, r) block pair of one update: sum_m G * B[l,m] B[m,r]
  const double2* A[MPS_MAX_D];   // B^[s][l, m] blocks, row-major Dl x Dm
  const double2* B[MPS_MAX_D];   // B^[s+1][m, r] blocks, row-major Dm x Dr
  int Dm[MPS_MAX_D];
  int gi[MPS_MAX_D];             // gate column (input basis index) per m
  double2* out[MPS_MAX_D];       // Theta'(c) at the (l, r) sub-block, per output charge c
  int ldo[MPS_MAX_D];            // row stride of Theta'(c)
  int go[MPS_MAX_D];             // gate row (output basis index) per c
  const double2* gate;           // gate block n = l - r, sn x sn row-major
  int sn;
  int Dl, Dr, nm, nc;
};
struct TileRef { int task; int ti; int tj; };

constexpr int kSvdSmem = 0;          // one CTA, the whole sector in shared memory
constexpr int kSvdCluster = 1;       // a thread-block cluster, data in L2, round-robin Jacobi
constexpr int kSvdClusterBlock = 2;  // a thread-block cluster, data in L2, block Jacobi staged in shared memory

struct SvdSector {            // one Theta(c): M = diag(rowscale) * Theta, m x n
  const double2* theta;       // row-major m x n
  const double* rowscale;     // m values (lambda of the left bond), or nullptr
  double2* work;              // cluster mode: M / R / R^dag, m x ld row-major (ld = n | 1)
  double2* uwork;             // cluster mode: Householder vector, m
  double* norms;              // cluster mode: 2n + K doubles (pivot norms, reference norms, Jacobi norms)
  int* order;                 // cluster mode: n + K ints (column permutation, singular value order)
  int* flags;                 // cluster mode: per-sweep rotation flags, then per-CTA pivot indices
  double* pivv;               // cluster mode: per-CTA pivot values, then two scalars
  double* sigma;              // out: min(m, n) values, descending
  double2* Y;                 // out: n x min(m, n) column-major right singular vectors
  int* status;                // out: Jacobi sweeps used, or -1 when not converged
  int m, n;
  int mode;                   // kSvdSmem, kSvdCluster or kSvdClusterBlock
  int groups;                 // block Jacobi: block pairs per CTA and round
  int staged;                 // block Jacobi: block pairs staged in shared memory at once
  double floor_rel;           // columns below floor_rel |M|_F are not rotated, their sigma is 0
                              // (0: the rounding-noise level 32 eps)
  double floor_abs;           // the same for an absolute level (0: none)
  int wide;                   // cluster mode, m < n: Jacobi on R2 of R^dag = Q2 R2 (K x K)
  double2* work2;             // wide: R2 / the Jacobi matrix, K x (K | 1) column-major
  double2* ytmp;              // wide: n x K, Q2 applied to the normalised columns
  // mixed-precision preconditioning (cluster mode, K >= the threshold; f32 == nullptr: off):
  float2* f32;                // the Jacobi matrix in FP32 stacked on V (identity), (jlen + K | 1) x K
  float* nrm32;               // K FP32 squared column norms
  double2* vd;                // K x K: the selected columns of V in FP64, then orthonormalised
  double2* gm;                // K x K: their Gram matrix, then its Cholesky factor
  double2* a1;                // jld x K: the Jacobi matrix times V, the start of the FP64 sweeps
  int* sel;                   // K + 1: selected columns, then their count
  int fp32_sweeps;            // limit of the FP32 sweeps
};

// Scratch layout of a batch of sector SVDs (cluster-mode sectors only need global scratch).
struct SvdScratchLayout {
  std::vector<int> mode;
  std::vector<int64_t> work_off, v_off, norm_off, ord_off, flag_off, piv_off, w2_off, yt_off;
  std::vector<int64_t> f32_off, n32_off, vd_off, gm_off, a1_off, sel_off;   // mixed precision (-1: off)
  std::vector<int> wide;
  int smem = 0;               // dynamic shared memory of the one-CTA kernel
  int64_t total = 0;
};
// Sectors that fit in shared memory run on the one-CTA kernel unless min(m, n) >= cluster_min_k
// (a cluster kernel then spreads them over several SMs; -1: the process setting
// mps_svd_cluster_min_k, off by default).
bool svd_layout(int ns, const int* m, const int* n, SvdScratchLayout& L, int cluster_min_k = -1);
int svd_cluster_min_k();
// Cluster sectors with min(m, n) >= this run FP32 Jacobi sweeps first and finish in FP64
// (0: every sector FP64 only); mps_svd_mixed_min_k sets it.
int svd_mixed_min_k();
int svd_mixed_sweeps();      // limit of the FP32 sweeps (mps_svd_mixed_sweeps)
// Points the cluster-mode scratch of sector k at base + the layout's offsets; sets S.mode.
void svd_fill_scratch(SvdSector& S, const SvdScratchLayout& L, int k, char* base);

struct SelectSector {         // one sector's spectrum as seen by the truncation
  const double* sigma;        // descending
  int k;                      // number of values (min(m, n))
};
struct SelectTask {           // one update: its sectors are [s0, s1) of the sector array
  int s0, s1;
  int chi;
  double cutoff;
};
struct SelectResult {         // per update
  double norm_all, norm_kept, trunc_err;
  double cut;                 // smallest kept singular value (0 if none)
  int band, n_candidates, status, pad;
};

struct GemmTask {             // C = alpha * A * B, A(i,k) = A[i*sar + k*sac], B(k,j) = B[k*sbr + j*sbc]
  const double2* A; const double2* B; double2* C;
  int M, N, K;
  int sar, sac, sbr, sbc, ldc;
  double alpha;
};
struct ScatterTask {          // B^[s+1][c, r] block: out[j*Dr + b] = conj(Y[(coff + b) + j*n])
  const double2* Y; double2* out;
  int n, coff, k, Dr;
  int64_t first;              // first flat element index of this task
};
struct LambdaTask {           // lambda[j] = sigma[j] * scale, j < k
  const double* sigma; double* lambda; int k; double scale;
};

// ---------------------------------------------------------------------------
// Device memory helpers.
// ---------------------------------------------------------------------------
struct DevBuf {
  void* p = nullptr; size_t bytes = 0;
  cudaError_t reserve(size_t want);
  void release();
};
struct PinnedBuf {
  void* p = nullptr; size_t bytes = 0;
  cudaError_t reserve(size_t want);
  void release();
};

struct Stats {
  int n_sectors = 0, n_triples = 0, max_sweeps = 0, tie_band = 0;
  double norm_all = 0, norm_kept = 0;
  int batch_sectors = 0, batch_sweeps_max = 0;   // over every update of the last call
  int64_t batch_sweeps_sum = 0;
  int64_t deflated_updates = 0, deflation_redos = 0;   // cut-estimate deflation, cumulative
};

struct KStat { int64_t launches = 0; double ms = 0, flops = 0, bytes = 0; };
// Work and device time of the last mps_dmrg call per kind (0: H_eff products, 1: environment
// updates, 2: Krylov vector work, 3: SVD, 4: other block contractions).
struct DmrgStats {
  int64_t matvecs = 0, restarts = 0;
  double ms[5] = {0, 0, 0, 0, 0}, flops[5] = {0, 0, 0, 0, 0};
  int64_t launches[5] = {0, 0, 0, 0, 0};
};
struct PendingTiming { int kind; cudaEvent_t a, b; bool pooled; };

// Kernel launches made by the library in this process (all handles).
void count_launch();

}  // namespace mps

struct mps_s {
  int L = 0, d = 0, N = 0, chi_max = 0, precision = 0;
  mps::ChargeRule rule;                   // U(1) or Z_n charge arithmetic (N is mod n for Z_n)
  cudaStream_t stream = nullptr;
  std::vector<mps::BondTable> bonds;      // L + 1
  std::vector<mps::SiteTable> sites;      // L
  std::vector<int> cur;                   // current slot (0/1) per site
  std::vector<char> dirty;                // site needs mps_set_site
  std::vector<int64_t> bond_cap;          // lambda capacity per bond
  std::vector<int64_t> lam_base;          // offset of each bond's lambda slot (doubles)
  std::vector<int64_t> site_cap;          // complex capacity of one site slot
  std::vector<int64_t> site_base;         // offset of slot 0 of each site (complex); slot 1 follows
  double* d_lambda = nullptr;
  double2* d_sites = nullptr;
  mps::DevBuf work;                       // per-update workspace
  mps::PinnedBuf pin_in, pin_out;         // staging of descriptors and results
  cudaEvent_t staged = nullptr;           // last upload out of pin_in has completed
  cudaStream_t side[mps::kSvdSideStreams] = {};     // side streams for concurrent SVD kernel groups
  cudaEvent_t fork = nullptr, join[mps::kSvdSideStreams] = {};
  std::string err;
  mps::Stats stats;
  bool profiling = false;
  mps::KStat kstat[MPS_K_COUNT];
  mps::DmrgStats dmrg_last;               // the last mps_dmrg call
  std::vector<mps::PendingTiming> pending;   // event pairs not yet read back
  std::vector<cudaEvent_t> event_pool;
  int* tc_flag = nullptr;                 // set by a tensor-core GEMM whose bounded wait expired
  std::vector<double> cut_est;            // per bond: smallest kept sigma of its last update (0: none)
  std::vector<int64_t> cut_call;          // per bond: the update call that recorded cut_est
  int64_t calls = 0;                      // update calls on this handle so far
  int sweep_limit = 40;                   // Jacobi sweep limit of this handle's update calls
  double chi_deflate = 3e-4;              // level of the deflation from a bond's previous chi cut (0: off)
  // CUDA graphs: the two launch phases of an update call are captured and replayed
  // through one executable graph each, updated in place while the topology holds
  bool graphs = false;
  bool capturing = false;
  cudaGraphExec_t gexec[2] = {nullptr, nullptr};
  int64_t graph_launches = 0, graph_updates = 0, graph_instantiations = 0;
  cudaEvent_t kind_ev[MPS_K_COUNT][2] = {};   // per-kind timing events used inside captured graphs
  // autotuning of the SVD tile shape per sector-size histogram
  bool autotune = false;

  double2* slot_ptr(int s, int slot) { return d_sites + site_base[s] + (slot ? site_cap[s] : 0); }
  double* lambda_ptr(int b) { return d_lambda + lam_base[b]; }
};

namespace mps {

// Kernel launchers (defined in the .cu files).
cudaError_t launch_theta(const ThetaTask* d_tasks, const TileRef* d_tiles, int n_tiles, cudaStream_t st);
// Sectors grouped by kernel and cluster size (a group is a contiguous run of the array).
struct SvdGroup { int kind, cl, smem, first, count; };
// Tile shape of the cluster SVD: target column-block width of the block-Jacobi kernel, the
// smallest cluster size tried, and the sector size (min(m, n)) from which a sector gets a
// cluster of 16 CTAs (the largest sectors of a layer set its critical path), and the sector
// size from which a sector runs the round-robin cluster kernel instead of the block-Jacobi one.
// The autotuner picks one per sector-size histogram.
struct SvdTune { int bw = 6; int cl_min = 2; int c16_min_k = 1 << 30; int rr_min_k = 1 << 30; };
constexpr int kTuneCands = 12;
// bw in {4, 6, 8, 12} x cl_min in {2, 4}; 16 CTAs from 512 or 256; round-robin from 512 or 256
inline SvdTune svd_tune_candidate(int k) {
  static const int bws[4] = {4, 6, 8, 12};
  SvdTune t;
  if (k >= 10) {
    t.rr_min_k = k == 10 ? 512 : 256;
    return t;
  }
  if (k >= 8) {
    t.c16_min_k = k == 8 ? 512 : 256;
    return t;
  }
  t.bw = bws[k & 3];
  t.cl_min = (k & 4) ? 4 : 2;
  return t;
}
// Orders `secs` into groups (costliest first inside each) and fills `groups`.
cudaError_t svd_group(std::vector<SvdSector>& secs, std::vector<SvdGroup>& groups,
                      const SvdTune& tune = SvdTune());
// The candidate mps_autotune_force set (true), or false when none is forced.
bool svd_forced_tune(SvdTune& t);
// Group 0 on st, group g > 0 on side[g-1] when n_side >= groups - 1; st then waits for all.
cudaError_t launch_svd_groups(const SvdSector* d_secs, const std::vector<SvdGroup>& groups, cudaStream_t st,
                              const cudaStream_t* side, int n_side, cudaEvent_t fork, const cudaEvent_t* join,
                              int max_sweeps = 40);

cudaError_t launch_select(const SelectSector* d_secs, const SelectTask* d_tasks, int n_tasks,
                          int* d_kept, SelectResult* d_res, cudaStream_t st);
cudaError_t launch_gemm(const GemmTask* d_tasks, const TileRef* d_tiles, int n_tiles, cudaStream_t st);

// TMA-fed tensor-core complex GEMM (k_tma.cu).  Operands live in "shadow tiles": 128 rows of
// 128 bytes each (16 KB), TF32 (a row holds 16 complex K as interleaved re, im floats) or BF16
// (a hi tile and a lo tile, a row holding 32 complex K).  An A tile row is one matrix row; a B
// tile holds 64 complex columns j as two rows each: 2j = conj(b_j), 2j + 1 = i conj(b_j), so
// that one real MMA of the interleaved K gives re and im of C in adjacent accumulator columns.
// All tiles of a call are slots of one buffer that a single 2-D tensor map describes.
constexpr int kShRows = 128;                  // rows of a shadow tile
constexpr int kShRowBytes = 128;              // bytes of a shadow tile row (the 128-byte swizzle span)
constexpr int64_t kShTileBytes = kShRows * kShRowBytes;
constexpr int kShTileN = 64;                  // complex columns of a B tile (= of an output tile)
inline int sh_kc(int precision) { return precision == MPS_BF16X3 ? 32 : 16; }   // complex K per tile
inline int sh_tiles_per_k(int precision) { return precision == MPS_BF16X3 ? 2 : 1; }   // hi (+ lo)
// One FP64 complex matrix into shadow tiles: element (i, k) = src[i * s_i + k * s_k];
// i runs over the rows (A) or the columns (B) of the operand.  Tile (it, kt) of the operand is
// slot tile0 + (it * kt_n + kt) * sh_tiles_per_k.  Rows and K beyond the matrix are zero.
struct ShadowTask {
  const double2* src;
  int64_t s_i, s_k;
  int n_i, K;                 // rows (A) / columns (B); complex K
  int64_t tile0;
  int kt_n;                   // K tiles per row tile
  int is_b;                   // 1: B-operand tile rows (two per column)
};
struct ShadowTile { int task, it, kt; };
cudaError_t launch_shadow(int precision, const ShadowTask* d_tasks, const ShadowTile* d_tiles, int n_tiles,
                          char* d_slots, cudaStream_t st);
// One 128 x 64 complex output tile of C = sum over K tiles (A tile a0 + kt) . (B tile b0 + kt):
// mode 0 stores it as complex64 (FP32) into C, mode 1 as complex128 scaled by alpha.
struct TmaJob {
  int64_t a0, b0;             // first A / B slot (K tiles follow, sh_tiles_per_k slots each)
  int kt_n;                   // K tiles (0: the product is zero)
  int M, N;                   // valid rows and complex columns of the tile
  int mode;
  float alpha;
  void* C;                    // element (0, 0) of the tile
  int64_t ldc;                // row stride of C in complex elements
};
// d_slots: the shadow buffer, n_slots tiles of kShTileBytes; *d_err = 1 when a bounded wait expires.
cudaError_t launch_tma_zgemm(int precision, const TmaJob* d_jobs, int n_jobs, const char* d_slots, int64_t n_slots,
                             int* d_err, cudaStream_t st);
// The gate mix of the Theta build on the tensor-core path: for one (l, r) pair with products
// T_i = B[s][l, m_i] B[s+1][m_i, r] (complex64, D_l x D_r, row stride ldt),
//   Theta'(c_o)[l, r] = sum_i G_n[go_o, gi_i] T_i      (FP64 into the Theta' workspace)
// and the same values as A-operand shadow tiles of the reassembly product (block (l, c_o):
// rows of l, K = the columns of Theta'(c_o), first K index coff_o).
struct MixTask {
  const float2* T[MPS_MAX_D];
  int gi[MPS_MAX_D];
  int nm;
  double2* out[MPS_MAX_D];
  int ldo[MPS_MAX_D];
  int go[MPS_MAX_D];
  int64_t sh0[MPS_MAX_D];         // reassembly A slots of block (l, c_o)
  int sh_ktn[MPS_MAX_D];          // K tiles of that block
  int coff[MPS_MAX_D];            // K offset of column 0 of r inside Theta'(c_o)
  int nc;
  const double2* gate;        // G_n, sn x sn row-major
  int sn;
  int Dl, Dr;
  int ldt;
};
cudaError_t launch_mix(int precision, const MixTask* d_tasks, int n_tasks, char* d_slots, cudaStream_t st);
cudaError_t launch_scatter(const ScatterTask* d_tasks, int n_tasks, int64_t n_elems, cudaStream_t st);
cudaError_t launch_lambda(const LambdaTask* d_tasks, int n_tasks, cudaStream_t st);

struct ExpectTask { const double2* blk; const double* lam; int Dl, Dm; double w; };
cudaError_t launch_expect(const ExpectTask* d_tasks, int n_tasks, double* d_partial, cudaStream_t st);
struct AmpStep { const double2* blk; int Dl, Dm; };
// Sequential pattern sampling: entry [site_off[s] + li * d + i] is the block (c, c - i) of site
// s for the li-th charge c of bond s (blk == nullptr when absent) and the index of c - i in
// bond s+1's table.
struct SampleEntry { const double2* blk; int Dl, Dm; int next; int pad; };
cudaError_t launch_sample(const SampleEntry* d_table, const int* d_site_off, int L, int d, int cap,
                          const double* d_uniforms, int n, int* d_configs, double* d_probs, cudaStream_t st);
// -sum lambda^2 ln lambda^2 over n values into *d_out (one CTA).
cudaError_t launch_entropy(const double* d_lambda, int n, double* d_out, cudaStream_t st);
cudaError_t launch_amplitude(const AmpStep* d_steps, int L, int n_cfg, double2* d_out, int chi_max,
                             cudaStream_t st);

// Shared-memory budget of the Jacobi kernel and its staging rule.
constexpr int kSvdThreads = 256;
constexpr int kSvdSmemMax = 200 * 1024;
int64_t svd_smem_need(int m, int n);
constexpr int kJacobiMaxSweeps = 40;
constexpr double kTieRel = 1e-11;
// Deflation of an update's SVDs: columns whose norm falls below kDeflateRel * cutoff * |M(c)|_F
// are left unrotated and reported as zero.  |M(c)|_F <= |sigma|_2 of the whole update, so they
// lie at least 100x below the cutoff threshold cutoff * |sigma|_2 and are discarded either way.
constexpr double kDeflateRel = 0.01;
// Deflation from the bond's previous cut: when chi set the last cut of a bond, columns below
// kChiDeflate * (the smallest singular value that update kept) are not resolved either.  The update is redone
// without it when its new cut falls below kChiVerify * that estimate, which keeps the level at
// or under 6e-4 of the actual cut (deflated values stay far below the cut; the kept values and
// vectors move by < 1e-13 on graded sectors).
constexpr double kChiDeflate = 3e-4;
constexpr double kChiVerify = 0.5;
// an update is redone when its cut falls below level / kChiGuard of the estimate (kChiGuard = 6e-4:
// an unresolved value then lies >= 1600x under the actual cut, whatever the level)
constexpr double kChiGuard = kChiDeflate / kChiVerify;

// GEMM tiling shared by the Theta build and the reassembly GEMM.
constexpr int kTile = 64;

}  // namespace mps
