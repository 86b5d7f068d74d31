/*
 * mps_gb300.h - C ABI of the GB300 U(1)-symmetric MPS two-site update library.
 *
 * The library keeps a U(1)-symmetric matrix product state on one GPU and applies
 * charge-conserving two-site gates to it by the block-sparse TEBD update of
 * arXiv:2303.11409, Sec. II: every bond index carries a right-charge
 * c^[k] = sum_{j>k} i_j, the Kronecker deltas of the U(1) amplitude formula force
 * c^[k-1] - c^[k] = i_k with c^[0] = N and c^[M] = 0, so a site tensor is a block
 * matrix without an explicit physical index, and a two-site update needs only
 * block-sparse SVDs of the submatrices Theta(c), each at most chi x chi.  On the
 * same sector machinery it runs two-site DMRG and TDVP (mps_dmrg, mps_tdvp), samples
 * occupation patterns (mps_sample), and supports Z_n charges (mps_create_zn,
 * mps_create_cyclic), several U(1) charges at once (mps_create_multi) and chain segments
 * for multi-rank runs (mps_create_segment).  Entry points that serve bookkeeping,
 * diagnostics or tuning say that the paper has no counterpart.
 *
 * Conventions used by every entry point
 *   - Sites are 0-based, s = 0..L-1.  Bond b (b = 0..L) sits left of site b, so
 *     site s joins bond s and bond s+1.  The charge of bond b is the number of
 *     particles on sites b..L-1; bond 0 carries N, bond L carries 0.
 *   - The state is stored right-canonical: B^[s] = Gamma^[s] lambda^[s+1] (the
 *     paper's Gamma/lambda pair), plus the Schmidt values lambda of every bond.
 *   - Block (l, m) of site s joins charge l of bond s and charge m of bond s+1;
 *     it exists iff 0 <= l - m <= d - 1 (the occupation of site s is l - m).
 *     Blocks are stored row-major, complex128 interleaved (re, im).
 *   - A two-site gate is given by its charge blocks G_n, n = 0..2(d-1); block n
 *     acts on the basis (i, n - i), i ascending over max(0, n-d+1)..min(d-1, n),
 *     i being the occupation of the left site; rows are outputs, columns inputs;
 *     blocks are concatenated in n order, each row-major complex128.
 *   - Host pointers passed in are read before the call returns; the caller keeps
 *     ownership.  The library owns all device memory of a handle.
 *   - Work is ordered on the handle's CUDA stream.  Results written to host
 *     pointers are complete when the call returns.
 *   - A handle is not thread-safe.  Every call returns an int status (below);
 *     mps_last_error() gives a message for the last failing call on a handle.
 */
#ifndef MPS_GB300_H
#define MPS_GB300_H

#include <stdint.h>

#if defined(__GNUC__)
#define MPS_API __attribute__((visibility("default")))
#else
#define MPS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mps_s* mps_t;

/* Status codes. */
#define MPS_OK        0   /* success */
#define MPS_EINVAL   -1   /* bad argument, size or state */
#define MPS_ECHARGE  -2   /* a charge outside [0, d-1] or an inconsistent charge table */
#define MPS_ENOMEM   -3   /* device or host allocation failed, or capacity exceeded */
#define MPS_ENOCONV  -4   /* a Jacobi SVD hit its sweep limit; the state was updated anyway */
#define MPS_ECUDA    -5   /* a CUDA runtime error */
#define MPS_ETIMEOUT -6   /* a bounded device wait expired */

/*
 * Precision modes of the sector GEMMs (the Theta' build and the reassembly product).
 * SVD, truncation and renormalisation are FP64 in all modes and follow the same
 * rules (the reduced modes only round the GEMM inputs); the observable error of
 * each mode against the FP64 result is stated with its tests.  A bounded-wait
 * expiry inside a tensor-core GEMM
 * is reported as MPS_ETIMEOUT by the update call that launched it, or, for the
 * reassembly product, by the next update call on the same handle or executor.
 */
#define MPS_FP64   0
#define MPS_TF32   1
#define MPS_BF16X3 2

/* Largest local dimension the library accepts. */
#define MPS_MAX_D 8

/*
 * mps_create - a product state |i_0 ... i_{L-1}> on the device.
 *   L             number of sites, >= 2
 *   d             local dimension, 2..MPS_MAX_D
 *   site_charges  host array of L occupations, each in [0, d-1]; N = their sum
 *                 (the paper's total charge, the boundary value c^[0] = N)
 *   precision     MPS_FP64, MPS_TF32 or MPS_BF16X3
 *   chi_max       largest bond dimension any later update may request, >= 1;
 *                 sizes the device arena (per bond min(chi_max, Hilbert bound))
 *   cuda_stream   cudaStream_t the handle works on (NULL = legacy default stream)
 * Errors: MPS_EINVAL, MPS_ECHARGE, MPS_ENOMEM, MPS_ECUDA.
 */
MPS_API int mps_create(mps_t* out, int L, int d, const int32_t* site_charges,
               int precision, int chi_max, void* cuda_stream);

/*
 * mps_create_segment - as mps_create, for a handle that holds only the sites
 * site_lo..site_hi-1 of the chain (0 <= site_lo < site_hi <= L): every other site keeps
 * the one element of its product-state block, so the arena is sized for the held sites
 * only.  An update, mps_set_site or mps_load that would grow a site outside the range
 * fails with MPS_ENOMEM (capacity exceeded) and leaves the state unchanged.  This is the
 * per-rank handle of a chain split into contiguous segments (Sec. II distributes
 * independent two-site updates across GPUs): a rank holds its own sites and one ghost
 * site beyond each cut.  Errors: as mps_create, and MPS_EINVAL for an empty or
 * out-of-range site range.
 */
MPS_API int mps_create_segment(mps_t* out, int L, int d, const int32_t* site_charges, int site_lo,
                               int site_hi, int precision, int chi_max, void* cuda_stream);

/*
 * mps_create_zn - like mps_create, for the cyclic group Z_n instead of U(1) (Sec. I names
 * more general Abelian symmetries; the block construction of Sec. II carries over): local
 * dimension d = n (2..MPS_MAX_D; mps_create_cyclic takes d < n), the physical index i
 * carries charge i mod n, bond b the right-charge (sum of the occupations right of it)
 * mod n, and every pair of charges forms
 * a site block (l, m) with i = (l - m) mod n.  Gate blocks for such a handle are the n blocks
 * q = 0..n-1 of the total charge (i + j) mod n, each n x n over the pairs (i, (q - i) mod n),
 * i ascending (rows outputs, columns inputs), concatenated row-major.  Every update, batch,
 * observable, amplitude and checkpoint call works on it; mps_create_segment and
 * mps_footprint_bytes are for U(1) handles only.  Errors as mps_create.
 */
MPS_API int mps_create_zn(mps_t* out, int L, int n, const int32_t* site_charges, int precision, int chi_max,
                          void* cuda_stream);

/*
 * mps_create_cyclic - a Z_n handle whose local dimension d may be below n (2 <= d <= n <=
 * 2^20; d = n is mps_create_zn).  The physical index i = 0..d-1 carries charge i mod n, bond
 * b the residue of the occupations right of it, and a site block (l, m) exists iff
 * (l - m) mod n < d; a Theta(c) then has as rows the left sectors l with (l - c) mod n < d,
 * in general not one run of the bond table (the update lists them and gathers their lambda).
 * Gate blocks are the residues q = (i + j) mod n reached by some pair, ascending, each over
 * its pairs (i, (q - i) mod n) with both entries below d, i ascending (rows outputs, columns
 * inputs), concatenated row-major.  A U(1)-conserving model (for example Bose-Hubbard with
 * n_max = d - 1) also conserves the particle number mod n; its U(1) gate blocks of totals
 * t = q, q + n, ... then sit in block q.  Calls as for mps_create_zn handles (Sec. I's
 * "more general Abelian" symmetries on the block construction of Sec. II).  Errors:
 * MPS_EINVAL (d or n out of range), as mps_create otherwise.
 */
MPS_API int mps_create_cyclic(mps_t* out, int L, int d, int n, const int32_t* site_charges, int precision,
                              int chi_max, void* cuda_stream);

/* mps_destroy - frees the handle and its device memory (after its stream drains); resource
 * management, no counterpart in the paper. */
MPS_API int mps_destroy(mps_t h);

/* mps_last_error - message of the last failing call on h ("" if none); owned by h.  No
 * counterpart in the paper. */
MPS_API const char* mps_last_error(mps_t h);

/* mps_info - L, d, N, chi_max and precision of a handle (any pointer may be NULL); N is the
 * boundary charge c^[0] of Sec. II. */
MPS_API int mps_info(mps_t h, int* L, int* d, int* N, int* chi_max, int* precision);

/*
 * mps_apply_gate2 - one two-site update on sites (site, site+1).
 *   gate_blocks   host complex128 gate blocks (layout above)
 *   chi           bond dimension cap for the new middle bond, 1..chi_max
 *   cutoff        keep only singular values > cutoff * |sigma|_2 (>= 0)
 *   trunc_err_out optional: discarded weight sum_disc sigma^2 / sum sigma^2
 * The update follows Sec. II: Theta'(c) = G . B^[s] B^[s+1] for every allowed
 * middle charge c, an FP64 SVD of diag(lambda^[s]) Theta'(c) per c, a global
 * top-chi truncation across all c (ties within 1e-11 sigma_max at the cut go to
 * the lower charge), then B^[s+1] = Y^dag_kept, B^[s] = Theta' Y_kept / |S_kept|
 * and lambda^[s+1] = S_kept / |S_kept|.  Within a sector the SVD does not resolve
 * singular values below 0.01 * cutoff * |M(c)|_F (at least 100x under the cutoff
 * threshold cutoff * |sigma|_2, so discarded in any case), nor, when chi set the cut
 * of the previous update of the same bond, below 3e-4 times that relative cut
 * (smallest kept value / |sigma|_2; the level is set by mps_set_chi_deflation) when that
 * cut was recorded by the previous update call on the handle, 30x lower when it is older:
 * their columns are not rotated and they count as zero.  When the new cut falls under
 * the applied level / 6e-4 of that previous one (half of it at 3e-4), the call redoes
 * that update's SVDs and the selection without the second level, so an unresolved value
 * always lies >= 1600x under the kept ones.
 * mps_deflation_stats counts updates that used the second level and those redone.
 * Errors: MPS_EINVAL, MPS_ENOMEM, MPS_ENOCONV (state updated), MPS_ECUDA.
 */
MPS_API int mps_apply_gate2(mps_t h, int site, const double* gate_blocks, int chi,
                    double cutoff, double* trunc_err_out);

/*
 * mps_apply_layer - n independent two-site updates on one handle in one set of
 * launches (Sec. II: two-site updates on disjoint pairs are independent and may
 * run in parallel).  sites[k] are left sites of pairwise disjoint pairs (no two differ by
 * less than 2); gate_blocks[k] are host gate blocks; chi and cutoff as above;
 * trunc_err_out (optional) receives n values.
 */
MPS_API int mps_apply_layer(mps_t h, int n, const int* sites, const double* const* gate_blocks,
                    int chi, double cutoff, double* trunc_err_out);

/*
 * mps_apply_gate2_batch - updates on several handles merged into shared launches.
 * Item k applies gates[k] at sites[k] of hs[k] with chis[k], cutoffs[k].  Items on
 * one handle must touch disjoint site pairs.  All handles must live on the current
 * device; work runs on hs[0]'s stream (the others' streams are joined first).
 * status_out[k] receives the per-item status; the return value is the first
 * non-OK item status, or MPS_OK.  Sec. II: two-site updates on disjoint pairs, here also
 * of different states, are independent and run as one batch.
 */
MPS_API int mps_apply_gate2_batch(int n, mps_t* hs, const int* sites, const double* const* gates,
                          const int* chis, const double* cutoffs, double* trunc_err_out,
                          int* status_out);

/*
 * mps_exec_t - an executor for merged updates across handles (serving): it owns the
 * workspace, staging buffers and stream that mps_exec_apply uses, so that handles can
 * come and go (requests admitted and completed) without the workspace moving.
 * mps_exec_create: cuda_stream as for mps_create.  mps_exec_destroy: after its stream drains.
 * mps_exec_apply: as mps_apply_gate2_batch, on the executor's stream and workspace;
 *   the handles may differ in L, d, chi_max (independent problems; Sec. II treats
 *   independent two-site updates as parallel work).
 */
typedef struct mps_s* mps_exec_t;
MPS_API int mps_exec_create(mps_exec_t* out, void* cuda_stream);
MPS_API int mps_exec_destroy(mps_exec_t ex);
MPS_API int mps_exec_apply(mps_exec_t ex, int n, mps_t* hs, const int* sites, const double* const* gates,
                           const int* chis, const double* cutoffs, double* trunc_err_out, int* status_out);

/*
 * mps_footprint_bytes - device memory a handle of (L, d, N, chi_max) holds (the arena
 * mps_create allocates: per bond min(chi_max, Hilbert bound) lambdas, two slots per
 * site of bond_cap(s) * bond_cap(s+1) complex numbers) and an upper bound of the
 * update workspace one of its Trotter layers needs (about 64 d chi^2 bytes per
 * update).  Host-only; used for admission by HBM footprint.  It follows the memory count
 * of Sec. II (every block at most chi x chi, bounded per bond by the charge-resolved
 * Hilbert dimension).
 */
MPS_API int mps_footprint_bytes(int L, int d, int N, int chi_max, int64_t* arena_bytes,
                                int64_t* layer_workspace_bytes);

/*
 * mps_expect - <O_site> of a diagonal one-site operator (U(1)-conserving one-site
 * operators are diagonal in the occupation basis).
 *   diag_op  host array of d real values O(i)
 *   out      host double: sum lambda^[s]_a^2 |B^[s]_{ab}|^2 O(l - m) over all blocks
 *            (the local canonical formula; lambda are the Schmidt values of Sec. II)
 */
MPS_API int mps_expect(mps_t h, int site, const double* diag_op, double* out);

/*
 * mps_amplitude - <i_0 ... i_{L-1}|psi>, the product of the one block per site the
 * charges select (the U(1) amplitude formula of Sec. II).
 *   config       host array of L occupations
 *   out_complex  host double[2] (re, im); 0 when sum(config) != N or an
 *                occupation is outside [0, d-1]
 */
MPS_API int mps_amplitude(mps_t h, const int32_t* config, double out_complex[2]);

/* mps_amplitude_batch - n amplitudes (the U(1) amplitude formula of Sec. II, one CTA per
 * configuration); configs is n x L row-major, out is n x 2. */
MPS_API int mps_amplitude_batch(mps_t h, int n, const int32_t* configs, double* out);

/*
 * mps_sample - n occupation patterns drawn from the state by sequential conditional
 * sampling (a follow-on of the U(1) amplitude formula of Sec. II, where the charges pick
 * one block per site).  In the right-canonical form the sites right of a bond form an
 * isometry, so the probability of a prefix i_0..i_{s-1} is |v_s|^2 with
 * v_s = B^[0][c_0, c_1] ... B^[s-1][c_{s-1}, c_s].  At site s every occupation i with a
 * block (c_s, c_s - i) has weight w_i = |v_s B^[s][c_s, c_s - i]|^2; the conditional
 * probability is w_i / sum_j w_j, and the drawn i is the first occupation, ascending,
 * whose cumulative conditional probability exceeds uniforms[k L + s]; v is then advanced
 * and rescaled to unit norm.
 *   uniforms     host array of n x L numbers in [0, 1), row-major (sample k, site s):
 *                the random draws are the caller's, so runs are reproducible
 *   configs_out  host int32 array of n x L occupations (row-major)
 *   probs_out    host array of n values (may be NULL): the product of the conditionals
 *                of each drawn pattern; on an exactly canonical, untruncated state it is
 *                |<pattern|psi>|^2
 * Work is one CTA per sample on the device; the call returns when the results are on the
 * host.  Errors: MPS_EINVAL (bad arguments, a site awaiting mps_set_site, a uniform
 * outside [0, 1), or a prefix whose continuations all have zero weight: that sample's
 * occupations from the failing site on are -1 and its probability 0), MPS_ENOMEM,
 * MPS_ECUDA.
 */
MPS_API int mps_sample(mps_t h, int n, const double* uniforms, int32_t* configs_out, double* probs_out);

/*
 * mps_bond_spectrum - the sectors of bond b (0..L): charges and dims ascending by
 * charge, and lambda values sector by sector (each sector descending): the Schmidt values
 * of Sec. II's canonical form, split by the bond charge.
 *   cap    capacity of charges/dims (sectors); lambda must hold the bond dimension
 *   n_out  number of sectors; if cap is too small nothing else is written and
 *          MPS_EINVAL is returned with n_out set
 */
MPS_API int mps_bond_spectrum(mps_t h, int bond, int32_t* charges, int32_t* dims, double* lambda,
                      int cap, int* n_out);

/*
 * mps_bond_entropy - the entanglement entropy of bond b (0..L) from its Schmidt values,
 * S_b = -sum_a lambda_a^2 ln lambda_a^2 over all sectors (natural log; lambda are the
 * Schmidt coefficients of the canonical form of Sec. II, unit 2-norm after every
 * update).  Computed on the device (one reduction kernel); *out is written when the
 * call returns.  Errors: MPS_EINVAL (bad bond, NULL out), MPS_ENOMEM, MPS_ECUDA.
 */
MPS_API int mps_bond_entropy(mps_t h, int bond, double* out);

/*
 * mps_get_site - the blocks B^[s][l, m] of site s (Sec. II's block matrix without an
 * explicit physical index) in (l ascending, m ascending) order.
 *   lcharges, mcharges  block labels (capacity cap_blocks)
 *   data                complex128 interleaved, blocks concatenated, each row-major
 *                       D_l x D_m (capacity cap_values complex numbers)
 *   n_blocks, n_values  sizes written (set even when a capacity is too small, in
 *                       which case MPS_EINVAL is returned and nothing else written)
 */
MPS_API int mps_get_site(mps_t h, int site, int32_t* lcharges, int32_t* mcharges, int cap_blocks,
                 double* data, int64_t cap_values, int* n_blocks, int64_t* n_values);

/*
 * mps_set_bond - replace the sector table and lambda of bond b (1..L-1).
 * mps_set_site - replace the blocks of site s; the blocks must be exactly the
 *   allowed (l, m) pairs of the current tables of bonds s and s+1, in (l, m)
 *   ascending order, with data laid out as in mps_get_site.
 * Together they load an arbitrary state (for checkpoints, tests and the ghost sites of
 * a segmented chain); set every bond first, then every site whose neighbouring bonds
 * changed.  mps_set_bond clears the deflation history of that bond only (the previous
 * cut an update of the bond would deflate from, see mps_apply_gate2); mps_set_site
 * keeps every bond's history.  The tables and blocks are those of Sec. II's block form.
 */
MPS_API int mps_set_bond(mps_t h, int bond, int n_sectors, const int32_t* charges, const int32_t* dims,
                 const double* lambda);
MPS_API int mps_set_site(mps_t h, int site, int n_blocks, const int32_t* lcharges, const int32_t* mcharges,
                 const double* data);

/*
 * mps_last_update_stats - diagnostics of the last update on h: counts of sectors,
 * (l,m,r) triples, Jacobi sweeps (max over sectors), ties resolved at the chi cut,
 * and the pre-renormalisation norm |S_all| and kept norm |S_kept|.
 * Any pointer may be NULL.  Diagnostics; no counterpart in the paper.
 */
MPS_API int mps_last_update_stats(mps_t h, int* n_sectors, int* n_triples, int* max_sweeps,
                          int* tie_band, double* norm_all, double* norm_kept);

/*
 * mps_set_chi_deflation - the second deflation level of the updates of h (see
 * mps_apply_gate2): singular values below level x the previous relative chi cut of the bond
 * (level / 30 when the previous update call on h did not record that cut) are left
 * unresolved, and an update whose new cut falls below the applied level / 6e-4 of that
 * estimate is redone without it, so an unresolved value always lies at least 1600x under the
 * kept ones.
 * level 0 turns the second level off; the default is 3e-4 (a redo when the cut halves); a
 * smaller level deflates less but redoes only after larger drops of the cut.  It applies to
 * the updates of h whichever handle's call (or executor) runs them.  MPS_EINVAL outside
 * [0, 6e-4].  A tuning of the SVD of Sec. II's update; no counterpart in the paper.
 */
MPS_API int mps_set_chi_deflation(mps_t h, double level);

/*
 * mps_deflation_stats - updates on h (cumulative) whose SVDs used the previous cut of
 * their bond as a deflation level, and how many of those were redone without it
 * (see mps_apply_gate2).  Either pointer may be NULL.  Diagnostics; no counterpart in the
 * paper.
 */
MPS_API int mps_deflation_stats(mps_t h, int64_t* deflated_updates, int64_t* redos);

/*
 * Kernel kinds reported by mps_kernel_stats.
 *   THETA   Theta'(c) build: sector GEMMs with the gate mixed in (Sec. II); in the TF32 /
 *           BF16x3 modes only the gate mix of the tensor-core products
 *   SVD     batched per-sector Jacobi SVD
 *   SELECT  global top-chi truncation across sectors
 *   LAMBDA, SCATTER, GEMM  reassembly of lambda, B^[s+1] and B^[s] (GEMM: FP64 mode)
 *   EXPECT, AMPLITUDE      measurements
 *   SAMPLE                 sequential pattern sampling (mps_sample; its work depends on the
 *                          drawn patterns and is counted as 0)
 *   TCGEMM  TF32 / BF16x3 modes: the tensor-core products of the Theta build and of the
 *           reassembly (flops of the complex products)
 *   SHADOW  TF32 / BF16x3 modes: operands converted into tensor-core shadow tiles
 */
#define MPS_K_THETA 0
#define MPS_K_SVD 1
#define MPS_K_SELECT 2
#define MPS_K_LAMBDA 3
#define MPS_K_SCATTER 4
#define MPS_K_GEMM 5
#define MPS_K_EXPECT 6
#define MPS_K_AMPLITUDE 7
#define MPS_K_SAMPLE 8
#define MPS_K_TCGEMM 9
#define MPS_K_SHADOW 10
#define MPS_K_COUNT 11

/*
 * mps_set_profiling - when on, every kernel launch of h is bracketed by CUDA events
 * on h's stream and its device time is accumulated per kind.
 * mps_kernel_stats - for one kind since the last reset: launches, summed device
 * milliseconds (0 unless profiling was on), and the algorithmic work of those
 * launches: flops (complex multiply-add = 8; SVD counted by the nominal
 * 4 (6 a b^2 + 20 b^3), a = max(m, n), b = min(m, n), per sector) and bytes
 * (compulsory reads + writes).  Synchronises h's stream.
 * mps_reset_kernel_stats - zeroes the counters of h.
 * mps_launch_count - kernels launched by this library in this process so far.
 * Measurement support; no counterpart in the paper.
 */
MPS_API int mps_set_profiling(mps_t h, int on);
MPS_API int mps_kernel_stats(mps_t h, int kind, int64_t* launches, double* ms, double* flops, double* bytes);
MPS_API int mps_reset_kernel_stats(mps_t h);
MPS_API int64_t mps_launch_count(void);

/*
 * mps_set_sweep_limit - the Jacobi sweep limit (1..40, default 40) of the update calls
 * whose owner or executor is h.  A sector that has not converged within it returns
 * MPS_ENOCONV and the state is updated with the last iterate (its singular values are
 * still exact column norms, but the vectors are not fully orthogonal).  A low limit is
 * how the non-convergence path is exercised in tests.  MPS_EINVAL outside 1..40.
 *
 * mps_tc_inject_stall - when on, the tensor-core GEMM kernels launched afterwards (in
 * any handle, and mps_zgemm_tc) issue no MMA, so their bounded mbarrier waits run out
 * after about 50 ms instead of 2 s: each such launch reports MPS_ETIMEOUT (an update
 * call returns it with the state unchanged).  For tests of the timeout path without
 * faulting or hanging the GPU; nothing is in flight when the kernel frees its tensor
 * memory.  The paper has no counterpart.
 */
MPS_API int mps_set_sweep_limit(mps_t h, int max_sweeps);
MPS_API int mps_tc_inject_stall(int on);

/*
 * mps_set_graphs - when on, each update call on h (mps_apply_gate2/_layer, and the
 * merged calls whose owner or executor is h) captures its two launch phases (upload,
 * Theta' build, SVD, top-chi selection and read-back; upload and reassembly) into CUDA
 * graphs and launches those: one executable graph per phase and handle, updated in
 * place (cudaGraphExecUpdate) when only launch parameters changed and instantiated
 * again when the topology changed.  Results are bit-identical to direct launches.
 * A handle on the legacy default stream (NULL) cannot be captured and keeps launching
 * directly.  Sec. II describes no graph mechanism; this is a launch-overhead measure.
 * mps_graph_stats - graph launches, in-place updates and instantiations on h so far.
 */
MPS_API int mps_set_graphs(mps_t h, int on);
MPS_API int mps_graph_stats(mps_t h, int64_t* launches, int64_t* updates, int64_t* instantiations);

/*
 * mps_set_autotune - when on, update calls on h choose the tile shape of the cluster
 * SVD (block-Jacobi column-block width 4, 6, 8 or 12 and smallest cluster 2 or 4 CTAs,
 * or clusters of 16 CTAs for sectors from min(m, n) = 512 or 256 up, where the device
 * places them; ten candidates) from a process-wide table keyed on the histogram of the
 * batch's large sectors
 * (octaves of min(m, n) holding at least 5% of the nominal SVD work, counts rounded to
 * powers of two).  The first batch with a new key whose nominal SVD work is at least
 * the tuning threshold (2e10 flops unless set) runs all ten shapes on its own inputs,
 * timed with CUDA events, and stores the fastest (the default shape, width 6 from
 * 2 CTAs, unless another beats it by more than 3%); its outputs come from the stored
 * shape.  Shapes differ only in rounding (the Jacobi pair order changes), so a tuned run
 * agrees with an untuned one to rounding, not bit for bit.
 * mps_autotune_stats - keys in the table, tuning runs made, and batches that reused a
 * stored shape (any pointer may be NULL).
 * mps_autotune_table - the table as text, one line per key; *len receives the length
 * without the terminator; buf may be NULL to query it (MPS_EINVAL if cap is too small).
 * mps_autotune_clear - empties the table.
 * mps_autotune_freeze - when frozen, batches with a key not in the table use the
 *   default shape and are not tuned (stored keys are still used).
 * mps_autotune_min_flops - the nominal SVD work (flops, >= 0) below which a batch is
 *   not tuned and uses the default shape.
 * mps_autotune_force - candidate 0..11 makes every update call of the process (and every
 *   mps_svd_sectors call) use that shape, whether or not autotuning is on (for tests and
 *   measurements); -1 ends it.  Candidates 0..7: width {4, 6, 8, 12}[k & 3], clusters
 *   from 2 << (k >> 2); 8 and 9: width 6 from 2 CTAs, 16-CTA clusters from min(m, n) =
 *   512 and 256; 10 and 11: the sectors from min(m, n) = 512 and 256 on the round-robin
 *   cluster kernel instead of the block-Jacobi one.  MPS_EINVAL for any other value.
 * Launch tuning of the per-sector SVDs of Sec. II; no counterpart in the paper.
 */
MPS_API int mps_set_autotune(mps_t h, int on);
MPS_API int mps_autotune_stats(int64_t* keys, int64_t* tuning_runs, int64_t* hits);
MPS_API int mps_autotune_table(char* buf, int cap, int* len);
MPS_API int mps_autotune_clear(void);
MPS_API int mps_autotune_freeze(int frozen);
MPS_API int mps_autotune_force(int candidate);
MPS_API int mps_autotune_min_flops(double flops);

/*
 * mps_last_batch_sweeps - Jacobi sweeps of the last update call on h over all of its
 * sectors: sector count, summed sweeps and the largest sweep count (any may be NULL).
 * Diagnostics of the per-sector SVDs of Sec. II; no counterpart in the paper.
 */
MPS_API int mps_last_batch_sweeps(mps_t h, int* n_sectors, int64_t* sweeps_sum, int* sweeps_max);

/*
 * mps_save - writes the current state of h (its charge rule: U(1), Z_n or several U(1)
 * charges; bond charge tables and Schmidt values, site blocks, and each bond's deflation
 * history) to the file `path` (created or truncated).  The file holds the
 * right-canonical B = Gamma lambda form the updates keep (Sec. II), so a handle
 * loaded from it continues the evolution bit for bit.  Synchronises h's stream.
 * Errors: MPS_EINVAL (NULL arguments, a site awaiting mps_set_site, I/O failure;
 * mps_last_error says which), MPS_ECUDA.
 *
 * mps_load - a new handle with the state stored by mps_save, on cuda_stream (as in
 * mps_create).  The stored charge rule, L, d, N, chi_max and precision are reused.  The
 * library owns the handle; free it with mps_destroy.  Errors: MPS_EINVAL (unreadable,
 * truncated or foreign file), MPS_ECHARGE (charge tables or blocks that violate the
 * charge structure), MPS_ENOMEM, MPS_ECUDA; *out is NULL on error.
 * The paper describes no checkpoint; this pair exists for long runs and serving.
 */
MPS_API int mps_save(mps_t h, const char* path);
MPS_API int mps_load(mps_t* out, const char* path, void* cuda_stream);

/*
 * mps_zgemm_tc - the tensor-core complex GEMM alone, on device memory:
 * C = A B with A (M x K), B (K x N), C (M x N) complex128 row-major (leading
 * dimensions lda >= K, ldb >= N, ldc >= N, in complex numbers).  precision is
 * MPS_TF32 (inputs rounded to FP32, then to TF32) or MPS_BF16X3 (each FP32-rounded
 * input split into two BF16 terms, three products accumulated).  The operands are
 * converted into shadow tiles in d_work, loaded by TMA (cp.async.bulk.tensor, 128-byte
 * swizzle) and multiplied by tcgen05.mma with FP32 accumulation in tensor memory, the
 * complex product lowered to one real GEMM; the result is converted to FP64 exactly.
 * This is the path the reduced-precision modes use for the sector GEMMs (Sec. II names
 * tensor cores for the GPU contraction).  d_work is device scratch of at least
 * mps_zgemm_tc_work_bytes(precision, M, N, K) bytes (-1 for invalid arguments).
 * Returns MPS_EINVAL for another precision or bad sizes, MPS_ETIMEOUT if a bounded wait
 * inside the kernel expired.  Synchronises cuda_stream.
 */
MPS_API int mps_zgemm_tc(int precision, int M, int N, int K, const double* d_A, int lda, const double* d_B,
                         int ldb, double* d_C, int ldc, void* d_work, int64_t work_bytes, void* cuda_stream);
MPS_API int64_t mps_zgemm_tc_work_bytes(int precision, int M, int N, int K);

/*
 * mps_fp64_peak_probe - measured FP64 FMA throughput of the current device in GFLOP/s
 * (independent FMA chains on every SM, about 70 ms).  The paper has no counterpart; the
 * SVD and GEMM kernels here are bound by this rate, so it is the denominator to read
 * their roofline against.  Allocates a small buffer on cuda_stream; synchronises it.
 */
MPS_API int mps_fp64_peak_probe(double* gflops, void* cuda_stream);

/*
 * mps_create_multi - a handle whose physical index i carries several U(1) charges at once,
 * the charge vector (phys_charges[i*ncomp + 0], ..., phys_charges[i*ncomp + ncomp-1]) (Sec. I
 * lists "more general Abelian" symmetries beside U(1); e.g. two conserved particle species).
 *   ncomp         1..4 charge components; every component >= 0; the vectors distinct and in
 *                 ascending lexicographic order of i
 *   site_indices  L physical indices in [0, d-1]: the initial product state
 *   precision     MPS_FP64, MPS_TF32 or MPS_BF16X3 (the sector GEMMs on the tensor cores, as
 *                 for mps_create; the listed rows and columns change no kernel)
 * Bond charges are the vector sums to the right of each bond, encoded as one int32 in mixed
 * radix (first component most significant; mps_charge_radix gives the radices, each more than
 * twice the largest bond value, so differences decode uniquely and the integer order is the
 * lexicographic one).  A block (l, m) exists iff l - m is a physical charge; the rows of a
 * Theta(c) are the left sectors l with l - c a physical charge (in general not one contiguous
 * run of the bond table; their lambdas are gathered before the SVD).  Gate and bond-term blocks
 * are the distinct pair totals q_i + q_j in ascending order, each over its pairs (i, j), i
 * ascending (rows outputs).  Every update, measurement, sampling and checkpoint call applies;
 * mps_dmrg and mps_tdvp are for single-U(1) handles.  Errors: MPS_EINVAL,
 * MPS_ECHARGE (a negative component, vectors not ascending, or encoded charges beyond int32),
 * MPS_ENOMEM.
 * mps_charge_radix - *ncomp and the radix of each component (radix may be NULL); 1 and 0 for
 * single-charge handles (the encoding of the vector charges above).
 */
MPS_API int mps_create_multi(mps_t* out, int L, int d, int ncomp, const int32_t* phys_charges,
                             const int32_t* site_indices, int precision, int chi_max, void* cuda_stream);
MPS_API int mps_charge_radix(mps_t h, int* ncomp, int32_t* radix);

/*
 * mps_charge_rule - the charge rule of a handle: *zn = n for a Z_n handle (0 otherwise),
 * *ncomp = the number of charge components of a several-U(1) handle (0 otherwise), and for
 * such a handle its d charge vectors into phys_charges (d x ncomp row-major, as passed to
 * mps_create_multi).  Any pointer may be NULL.  A handle from mps_load reports the rule it
 * was saved with.  (Sec. I's symmetry groups: U(1), Z_n, products of U(1).)
 */
MPS_API int mps_charge_rule(mps_t h, int* zn, int* ncomp, int32_t* phys_charges);

/*
 * mps_dmrg - two-site DMRG sweeps on the state of h (ground states of the U(1) chains the
 * paper cites DMRG for, Sec. I, on the block structure of Sec. II: the two-site wave function
 * is split by its middle charge into the Theta(c) blocks of the TEBD update, each with its own
 * SVD, truncated globally as mps_apply_gate2 does).
 *   bond_terms   L-1 host pointers; bond_terms[k] is the Hermitian two-site term h_{k,k+1}
 *                of H = sum_k h_{k,k+1} as charge blocks in the gate layout (block n over the
 *                pairs (i, n - i), i ascending, rows outputs; interleaved complex128, the
 *                sum over n of s_n^2 complex numbers, s_n the size of block n); read
 *                during the call only
 *   n_sweeps     sweeps; a sweep is a right-moving pass over the pairs (0,1) .. (L-2,L-1)
 *                and a left-moving pass back (2 (L-1) local steps)
 *   chi, cutoff  the truncation of every local step (the rule of mps_apply_gate2)
 *   lanczos_dim  Krylov dimension of one Lanczos cycle (2..63); cycles restart from the
 *                Ritz vector until the residual |H_eff psi - E psi| <= tol max(1, |E|)
 *   energies     out (may be NULL): the Lanczos eigenvalue of every local step, in order;
 *                energies_cap >= n_sweeps * 2 (L-1) when given
 *   n_energies   out: local steps done
 * The state must be right-canonical (any state the update calls produce, or a product
 * state) and h an FP64 U(1) handle.  On return the state is right-canonical again with every
 * lambda the Schmidt values of its bond (an inverse-free left-to-right pass), so the
 * observables, sampling and update calls apply to it.  MPS_ENOCONV when a Lanczos
 * or a Jacobi SVD stopped at its limit (the state is updated with the last iterate),
 * MPS_EINVAL for bad arguments, a TF32/BF16x3 or Z_n handle, or a site set with mps_set_site
 * but not yet valid; MPS_ENOMEM when a bond outgrows the handle's chi_max capacity.
 * mps_dmrg_stats reports, for the last call, per kind (0: H_eff products, 1: environment
 * updates, 2: Krylov vector work, 3: SVD, 4: other block contractions) the launches, the
 * device milliseconds (with mps_set_profiling on) and the algorithmic flops; mps_dmrg_counts
 * the H_eff products and Lanczos cycles (diagnostics, no counterpart in the paper).
 */
MPS_API int mps_dmrg(mps_t h, const double* const* bond_terms, int n_sweeps, int chi, double cutoff,
                     int lanczos_dim, double tol, double* energies, int energies_cap, int* n_energies);
MPS_API int mps_dmrg_stats(mps_t h, int kind, int64_t* launches, double* ms, double* flops);
/*
 * mps_tdvp - second-order two-site TDVP (time-dependent variational principle) time steps on
 * the state of h, the real-time counterpart of mps_dmrg on the same environments and H_eff (the
 * paper names no time-evolution scheme beyond TEBD, Sec. I; this is the standard two-site one):
 * a step of length dt is a right-moving and a left-moving pass of dt/2; each pair is evolved
 * by exp(-i dt/2 H_eff) (a Krylov exponential on the device: Lanczos basis of krylov_dim
 * vectors, 2..40, the tridiagonal's eigenpairs by Jacobi rotations; the step is split into
 * substeps until the error estimate |beta y_last| <= tol), split per middle charge with the
 * truncation of mps_apply_gate2, and the new centre site evolved backward by exp(+i dt/2
 * H_eff^(1)) with its one-site effective Hamiltonian, except at the turn.  Arguments, the
 * storage form on entry and exit, and the errors are those of mps_dmrg; energies receives
 * <psi|H_eff|psi> of the pair before each of the 2 (L-1) n_steps forward evolutions; mps_dmrg_stats
 * reports the call's work (kind 0 counts both the two-site and the one-site H_eff products).
 */
MPS_API int mps_tdvp(mps_t h, const double* const* bond_terms, int n_steps, double dt, int chi, double cutoff,
                     int krylov_dim, double tol, double* energies, int energies_cap, int* n_energies);
MPS_API int mps_dmrg_counts(mps_t h, int64_t* matvecs, int64_t* restarts);

/*
 * mps_plan_sectors - the integer sector planner alone (host code, no GPU needed).
 * Given the charge tables of bonds s, s+1, s+2 (ascending charges), it lists every
 * compatible (l, m, r) with 0 <= l-m <= d-1 and 0 <= m-r <= d-1, and every
 * candidate middle charge c with its Theta(c) size: rows = sum of D_l over
 * c <= l <= c+d-1, cols = sum of D_r over c-d+1 <= r <= c (Sec. II).
 *   triples     out, 3 ints per triple (l, m, r), lexicographic ascending
 *   sectors     out, 3 ints per sector (c, rows, cols), c ascending
 *   n_triples, n_sectors  sizes written; MPS_EINVAL if a capacity is too small
 */
MPS_API int mps_plan_sectors(int d, int nl, const int32_t* lc, const int32_t* ld,
                     int nm, const int32_t* mc, const int32_t* md,
                     int nr, const int32_t* rc, const int32_t* rd,
                     int32_t* triples, int cap_triples, int* n_triples,
                     int32_t* sectors, int cap_sectors, int* n_sectors);

/*
 * mps_plan_sectors_rule - the sector planner of mps_plan_sectors for every charge rule a handle
 * can have (host code, no GPU needed): U(1) (zn = 0, ncomp = 0, as mps_plan_sectors), Z_n
 * (zn = n >= d, as mps_create_zn and mps_create_cyclic) and several U(1) charges (ncomp >= 1,
 * as mps_create_multi).
 * Sec. II's Kronecker deltas give the blocks: (l, m) is a site block iff l - m is the charge of
 * a physical index (taken mod n for Z_n, as a vector for several charges), and Theta(c) has as
 * rows the left sectors l with l - c such a charge and as columns the right sectors r with
 * c - r one.
 *   phys_charges  (ncomp >= 1) d x ncomp row-major charge vectors, ascending, components >= 0
 *   radix         (ncomp >= 1) the mixed radix of the encoded bond charges (first component
 *                 most significant; mps_charge_radix of a handle gives it); every component of a
 *                 physical or bond charge must lie below radix / 2, else MPS_ECHARGE
 *   lc, mc, rc    ascending bond charges (residues in [0, n-1] for Z_n, encoded for ncomp >= 1)
 *   triples       out, 3 ints per (l, m, r), lexicographic in the tables' order
 *   sectors       out, 5 ints per candidate middle charge: (c, rows, cols, row sectors,
 *                 column sectors), c ascending
 *   lists         out, per sector its row sector charges then its column sector charges
 *   n_triples, n_sectors, n_lists  sizes written; MPS_EINVAL if a capacity is too small, for
 *                 zn < d or zn > 2^20, or for zn and ncomp both set
 */
MPS_API int mps_plan_sectors_rule(int d, int zn, int ncomp, const int32_t* phys_charges, const int32_t* radix,
                     int nl, const int32_t* lc, const int32_t* ld,
                     int nm, const int32_t* mc, const int32_t* md,
                     int nr, const int32_t* rc, const int32_t* rd,
                     int32_t* triples, int cap_triples, int* n_triples,
                     int32_t* sectors, int cap_sectors, int* n_sectors,
                     int32_t* lists, int cap_lists, int* n_lists);

/*
 * mps_gate_layout - the two-site gate (and bond-term) layout of a charge rule (host code, no
 * GPU needed): the sizes s_k of its blocks in layout order into sizes (capacity cap; may be
 * NULL), their number *n_blocks and the flattened length sum_k s_k^2 in complex numbers that
 * every gate passed to an update of such a handle holds.  U(1) (zn = 0, ncomp = 0): blocks
 * n = 0..2(d-1) over (i, n - i); Z_n (zn = n >= d): the residues q = (i + j) mod n some pair
 * reaches; several U(1) charges (ncomp >= 1, phys_charges as for mps_create_multi): the distinct
 * totals q_i + q_j, lexicographic.  The charge of a pair is the sum of Sec. II's local charges.
 * Errors: MPS_EINVAL (bad arguments, cap too small), MPS_ECHARGE (charge vectors negative or
 * not ascending).
 */
MPS_API int mps_gate_layout(int d, int zn, int ncomp, const int32_t* phys_charges, int32_t* sizes, int cap,
                            int* n_blocks, int64_t* length);

/*
 * mps_svd_sectors - the batched per-sector SVD kernel alone, on device memory
 * (one-sided Jacobi in FP64; Sec. II: the local update needs one SVD per charge block).
 * For each sector k it decomposes M_k = diag(rowscale_k) A_k, A_k being the
 * m_k x n_k row-major complex128 matrix at d_mats + mat_off[k] (in complex
 * numbers), rowscale_k the m_k doubles at d_rowscale + row_off[k] (NULL = 1):
 *   d_sigma + sig_off[k]   min(m_k, n_k) singular values, descending
 *   d_y + y_off[k]         the right singular vectors as an n_k x min(m_k,n_k)
 *                          column-major complex128 matrix Y (M = X S Y^dag)
 *   d_status[k]            Jacobi sweeps used, or -1 if not converged
 * mat_off, row_off, sig_off, y_off, m, n are host int64/int arrays of length
 * n_sectors; d_work is device scratch of work_bytes bytes, at least
 * mps_svd_work_bytes(...) for the same sizes.
 */
MPS_API int64_t mps_svd_work_bytes(int n_sectors, const int* m, const int* n);
MPS_API int mps_svd_sectors(int n_sectors, const int* m, const int* n,
                    const double* d_mats, const int64_t* mat_off,
                    const double* d_rowscale, const int64_t* row_off,
                    double* d_sigma, const int64_t* sig_off,
                    double* d_y, const int64_t* y_off,
                    int* d_status, void* d_work, int64_t work_bytes, void* cuda_stream);

/*
 * mps_svd_mixed_min_k - sectors of the cluster SVD kernels with min(m, n) >= min_k (default 192;
 * 0: none) first run one-sided Jacobi sweeps in FP32 on the Jacobi matrix stacked on the
 * identity, which accumulates the rotations V; V is then made unitary in FP64 (one Cholesky
 * QR) and the FP64 sweeps start from the Jacobi matrix times V, converging in 2-3 sweeps.
 * Results meet the same FP64 accuracy; FP32 runs at 61x the FP64 rate on this part.  A process
 * setting, read when an update call or mps_svd_sectors lays out its scratch (more scratch per
 * such sector: about 8 (jlen + K) K + 48 K^2 bytes).  MPS_EINVAL for min_k < 0.  A tuning of
 * the per-sector SVDs of Sec. II; no counterpart in the paper.
 */
MPS_API int mps_svd_mixed_min_k(int min_k);
/* mps_svd_mixed_sweeps - the limit of those FP32 sweeps (1..40, default 8: on the chi = 2048 layer 6-10
 * FP32 sweeps minimise the time; the FP64 sweeps finish either way); MPS_EINVAL outside.  Tuning;
 * no counterpart in the paper. */
MPS_API int mps_svd_mixed_sweeps(int max_sweeps);
/* mps_svd_cluster_min_k - sectors with min(m, n) >= min_k run on the cluster SVD kernels even when
 * they fit in one CTA's shared memory (spreading a batch of few sectors over more SMs); 0 (the
 * default): only sectors that do not fit.  A process setting read when mps_svd_sectors or an
 * update call lays out its scratch; mps_dmrg picks its own threshold per step.  MPS_EINVAL for
 * 0 < min_k < 16 or min_k < 0.  Tuning; no counterpart in the paper. */
MPS_API int mps_svd_cluster_min_k(int min_k);

/*
 * mps_svd_sectors_noalloc - the batched sector SVD of mps_svd_sectors for callers
 * that must not allocate device memory.  The paper has no counterpart to this
 * entry point; it exists for callers whose device memory is owned by someone
 * else: code running under a framework's memory manager that reserves the whole
 * budget, hot loops where the implicit device synchronisation of cudaMalloc and
 * cudaFree is not acceptable, and callers that are not allowed to hand the
 * library a scratch buffer at all.
 *   Arguments, layouts and outputs are those of mps_svd_sectors, without d_work
 *   and work_bytes.  Instead of caller scratch it uses one file-scope device
 *   array of MPS_NOALLOC_SCRATCH_BYTES bytes that every GPU which loads the
 *   library holds until the process exits.
 *   Limit: mps_svd_work_bytes() of the batch must not exceed
 *   MPS_NOALLOC_SCRATCH_BYTES; larger batches are rejected with MPS_ENOMEM before
 *   anything runs (split the batch, or use mps_svd_sectors).
 *   The first call on a device looks up the array's device address with that
 *   device current; make that first call before any stream capture.
 *   It calls no cudaMalloc, cudaFree or other allocating routine.  All calls
 *   share the one array, and each call overwrites every part of it that it reads,
 *   so nothing needs clearing between calls; calls that overlap on the GPU (other
 *   streams, other host threads) race on it and must be serialised by the caller.
 *   Like mps_svd_sectors it synchronises cuda_stream before returning.
 */
#define MPS_NOALLOC_SCRATCH_BYTES (16 * 1024 * 1024)
MPS_API int mps_svd_sectors_noalloc(int n_sectors, const int* m, const int* n,
                                    const double* d_mats, const int64_t* mat_off,
                                    const double* d_rowscale, const int64_t* row_off,
                                    double* d_sigma, const int64_t* sig_off,
                                    double* d_y, const int64_t* y_off,
                                    int* d_status, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* MPS_GB300_H */
