/*
 * polar_express.h -- C ABI of the GB300 (sm_103a) Polar Express library.
 *
 * The library computes the polar factor polar(G) = U V^T of G = U S V^T
 * (Eq. matrixsign) with the Polar Express method: Frobenius normalisation
 * followed by T odd polynomial steps X <- a_t X + (b_t A + c_t A^2) X with
 * A = X X^T on the short side (Alg. 1, online stage; Sec. 3.5 Horner form).
 * The per-step coefficients come from the greedy minimax construction of
 * Thm. 1 (Alg. 1, offline stage), solved on the host in FP64.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Return value: a pe_status. On any status other than PE_OK a thread-local
 *    message is available from pe_last_error().
 *  - Argument errors (PE_EINVAL, PE_EUNSUPPORTED) are detected synchronously,
 *    before anything is enqueued; device buffers are then left untouched.
 *  - Device entry points are asynchronous with respect to the host: they
 *    enqueue work on `stream` (a cudaStream_t passed as void*; NULL is the
 *    legacy default stream) and return. Failures that only the device can
 *    see (a bounded wait that expired, a non-finite norm) are latched in a
 *    per-device status word and reported (then cleared) by pe_sync_status(),
 *    as PE_ETIMEOUT or PE_ECUDA.
 *  - Matrices are dense row-major: element (i, j) of an m x n matrix with
 *    leading dimension ld lives at base[i * ld + j].
 *  - Workspace is owned by the library: a per-device pool that grows on
 *    demand (cudaMalloc, never inside a stream capture) and is freed by
 *    pe_release(). Calls that would allocate while `stream` is capturing
 *    fail with PE_EINVAL; warm the call up once before capturing it.
 *  - Calls that share workspace are serialised by the library's host lock;
 *    concurrent calls on different streams of one device therefore also
 *    serialise their enqueue, and their kernels must not overlap on the
 *    device (keep them on one stream or order the streams).
 */
#ifndef POLAR_EXPRESS_H
#define POLAR_EXPRESS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PE_OK = 0,
    PE_EINVAL = 1,        /* bad argument */
    PE_ENOMEM = 2,        /* workspace allocation failed */
    PE_ECUDA = 3,         /* a CUDA runtime/driver call failed, or a non-finite norm */
    PE_ENOCONV = 4,       /* the Remez iteration hit its iteration cap */
    PE_ETIMEOUT = 5,      /* a bounded device wait expired (results invalid) */
    PE_EUNSUPPORTED = 6   /* valid request that the library or the device does not support */
} pe_status;

/* Arithmetic of the online stage. */
typedef enum {
    PE_FP32 = 0,   /* plain method: FP32 operands, FP32 FMA accumulation (no TF32) */
    PE_BF16 = 1,   /* BF16 tensor-core operands, FP32 accumulation, FP32 master X */
    PE_BF16X3 = 2  /* split BF16: x = hi + lo, three BF16 products per k-step
                      (hi*hi + hi*lo + lo*hi), FP32 accumulation */
} pe_dtype;

/* Element type of the caller's matrices. */
typedef enum {
    PE_IO_FP32 = 0,
    PE_IO_BF16 = 1
} pe_io_type;

/* Flags for pe_coeffs_ex. */
#define PE_SAFETY_SKIP_LAST 1u  /* leave the final row without the safety factor
                                   (App. G: it may be omitted in the last step) */

/* Library version as 10000*major + 100*minor + patch. */
int pe_version(void);

/*
 * pe_coeffs -- offline stage: the greedy minimax coefficient table.
 *
 * Defined by Thm. 1 (Eq. greedy, Eq. newbounds) with the stabilisations of
 * Sec. 3.4 / App. G and the offline code of App. A:
 *   l_1 = l, u_1 = 1; for t = 1..T:
 *     p_t = minimax odd polynomial of `degree` for x -> 1 on
 *           [max(l_t, kappa u_t), u_t]  (degree 5: Remez of Alg. 3, App. F;
 *           degree 3: closed form Eq. deg3_solution);
 *     p_t <- p_t * 2 / (p_t(l_t) + max p_t on [l_t, u_t])   (recentring);
 *     l_{t+1} = p_t(l_t), u_{t+1} = 2 - l_{t+1};
 *   then every row that did not come from the l/u -> 1 shortcut (App. F) is
 *   replaced by p_t(x / safety).
 * kappa = 0.02407327424182761 for degree 5 (App. A), 0.1 for degree 3
 * (Alg. 1's u/10).
 *
 *   degree  3 or 5.
 *   l       lower bound on the normalised singular values, 0 < l <= 1.
 *   T       number of steps, 1 <= T <= 64.
 *   safety  >= 1; 1 disables the safety factor (the paper uses 1.01).
 *   coeffs  out, host, caller-owned, 3*T doubles: row t is (a_t, b_t, c_t) of
 *           p_t(x) = a_t x + b_t x^3 + c_t x^5 (c_t = 0 for degree 3).
 *   bounds  out, host, caller-owned, 2*(T+1) doubles (l_t, u_t) before the
 *           safety factor, or NULL.
 * Pure host FP64 code, deterministic and reproducible bit for bit (no FMA
 * contraction; fixed elimination order in the 4x4 solves).
 * Errors: PE_EINVAL for arguments out of range or NULL coeffs, PE_ENOCONV if
 * a Remez solve does not converge in 100 iterations.
 */
int pe_coeffs(int degree, double l, int T, double safety, double* coeffs, double* bounds);

/*
 * pe_coeffs_ex -- pe_coeffs with the remaining knobs of the offline stage.
 *   cushion      kappa; a negative value selects the default for `degree`,
 *                0 disables cushioning (the pure greedy optimum of Thm. 1).
 *   flags        PE_SAFETY_SKIP_LAST or 0.
 *   remez_iters  out, nullable: T ints, Remez iterations used per step
 *                (0 for the shortcut and for degree 3).
 */
int pe_coeffs_ex(int degree, double l, int T, double safety, double cushion, unsigned flags,
                 double* coeffs, double* bounds, int* remez_iters);

/*
 * pe_polar -- online stage for one matrix, in place.
 *
 * Computes X_T = p_T(...p_1(X_0)) with X_0 = G / (1.01 ||G||_F + 1e-7)
 * (App. A online code) taken on the short side (transposed when m > n, so
 * that A = X X^T is min(m,n) x min(m,n); App. A, Sec. H), and each step
 * A = X X^T, B = b_t A + c_t A^2, X <- a_t X + B X (Sec. 3.5).
 *
 *   X       in/out, device, m x n row-major contiguous FP32 (ld = n). On
 *           return (stream order) it holds X_T ~ polar(G).
 *   m, n    >= 1.
 *   table   host, T rows of (a, b, c) doubles (from pe_coeffs or any fixed
 *           table such as Newton-Schulz (15/8, -10/8, 3/8)); cast to FP32.
 *   T       1..64.
 *   dtype   a pe_dtype.
 *   stream  cudaStream_t as void*.
 * Errors: PE_EINVAL (NULL pointers, sizes, T, dtype, non-finite table),
 * PE_ENOMEM, PE_ECUDA, PE_EUNSUPPORTED (device is not sm_103).
 */
int pe_polar(void* X, int64_t m, int64_t n, const double* table, int T, int dtype, void* stream);

/*
 * pe_polar_ex -- pe_polar with explicit layout, element type and the
 * normalisation constants.
 *   ld          leading dimension in elements, >= n.
 *   io_type     PE_IO_FP32 or PE_IO_BF16 (X is read and written in that type;
 *               the iteration itself runs in `dtype`).
 *   norm_scale  multiplies ||G||_F (App. A code: 1.01; Alg. 1: 1.0).
 *   norm_eps    added to the scaled norm (App. A code: 1e-7; Alg. 1: 1e-2).
 */
int pe_polar_ex(void* X, int64_t m, int64_t n, int64_t ld, int io_type,
                const double* table, int T, int dtype,
                double norm_scale, double norm_eps, void* stream);

/*
 * pe_polar_batched -- online stage for a list of matrices of uneven shapes
 * (all of a model's Muon parameters), in place.
 *
 * Same mathematics as pe_polar applied to each X[i] independently. The
 * matrices are processed together: one grouped normalisation launch, then per
 * polynomial step one persistent grouped launch (BF16 paths) that runs the
 * Gram, A^2 and update tiles of every matrix with per-matrix readiness
 * counters, all inside a CUDA graph cached by the library under the key
 * (pointers, shapes, T, dtype, table). The first call with a new key tunes
 * the tile schedule and captures the graph (it synchronises `stream` once);
 * later calls replay the graph.
 *
 *   X       host array of `count` device pointers, each m[i] x n[i] row-major
 *           contiguous FP32, in/out.
 *   m, n    host arrays of `count` sizes (>= 1).
 *   count   1..4096.
 *   table, T, dtype, stream as for pe_polar.
 * Errors: as pe_polar; a bounded readiness wait that expires on the device is
 * reported as PE_ETIMEOUT by pe_sync_status() or the next call.
 */
int pe_polar_batched(void* const* X, const int64_t* m, const int64_t* n, int count,
                     const double* table, int T, int dtype, void* stream);

/*
 * pe_polar_batched_ex -- pe_polar_batched with the element type and the
 * normalisation constants of pe_polar_ex, and control over the plan:
 *   flags  bit 0 (PE_BATCH_NO_GRAPH): enqueue kernels directly, no graph;
 *          bit 1 (PE_BATCH_NO_TUNE): keep the default tile schedule;
 *          bit 2 (PE_BATCH_PHASED): three grouped launches per step (Gram,
 *          A^2, update) instead of one persistent launch.
 */
#define PE_BATCH_NO_GRAPH 1u
#define PE_BATCH_NO_TUNE 2u
#define PE_BATCH_PHASED 4u
int pe_polar_batched_ex(void* const* X, const int64_t* m, const int64_t* n, int count, int io_type,
                        const double* table, int T, int dtype,
                        double norm_scale, double norm_eps, unsigned flags, void* stream);

/*
 * pe_sync_status -- synchronise `stream` and report (then clear) the device
 * status word of the current device: PE_OK, PE_ETIMEOUT (a bounded readiness
 * or pipeline wait expired), PE_ECUDA (a kernel error, a non-finite norm, or
 * mismatched tensor-memory bases in a 2-SM pair).
 */
int pe_sync_status(void* stream);

/* Host-buffer form of pe_polar_batched (FP32, fixed normalisation 1.01 /
 * 1e-7): Hin[i] (read) and Hout[i] (written) are host m[i] x n[i] row-major
 * FP32 matrices; pinned memory (cudaHostAlloc / torch pin_memory) lets the
 * copies run asynchronously at full link bandwidth. The library keeps device
 * staging buffers per shape set (4 sets, LRU; pe_release frees them) and
 * pipelines: the matrices are cut into `ngroups` contiguous groups of about
 * equal bytes (0 = automatic: min(count, 6)); group
 * g's host->device copies run on one internal stream, its grouped compute on
 * `stream` once they have landed, its device->host copies on a second
 * internal stream, so copies in both directions overlap compute of other
 * groups. All work is ordered after what is already queued on `stream`, and
 * `stream` waits for the last copy, so synchronising `stream` means Hout is
 * complete. Calls that share a shape set must not overlap in time (they share
 * the staging buffers). Errors: as pe_polar_batched, PE_ENOMEM for the
 * staging buffers. Results are those of pe_polar_batched on the same data. */
int pe_polar_batched_host(const void* const* Hin, void* const* Hout, const int64_t* m, const int64_t* n, int count,
                          const double* table, int T, int dtype, int ngroups, void* stream);

/* Number of this library's kernels enqueued (directly or inside replayed
 * graphs) on the calling process since load; for launch accounting. */
int64_t pe_launch_count(void);

/*
 * Tracing: per-kernel device time. While tracing is on, device calls enqueue
 * their kernels directly (no graph) and bracket every launch with a pair of
 * CUDA events recorded on the call's stream.
 *   pe_trace_enable(1) clears the record and starts tracing; (0) stops it.
 *   pe_trace_read synchronises the recorded events and writes, for kernel
 *   kind k < nkinds, launches[k] and ms[k] (total device milliseconds):
 *     0 norm partials, 1 prepare, 2 FP32 Gram, 3 FP32 square, 4 FP32 update,
 *     5 tcgen05 fused step, 6 tcgen05 Gram phase, 7 tcgen05 square phase,
 *     8 tcgen05 update phase.
 *   Returns PE_EINVAL for NULL outputs or nkinds < 1.
 */
#define PE_TRACE_KINDS 9
int pe_trace_enable(int on);
int pe_trace_read(int64_t* launches, double* ms, int nkinds);

/* Message for the last non-OK status returned on this thread ("" if none). */
const char* pe_last_error(void);

/* Free all workspace and cached plans of all devices. Safe to call anytime
 * the library's work has completed. */
void pe_release(void);

/*
 * pe_debug_set -- test hooks, off by default.
 *   key 1: withhold the readiness signal of matrix `value` in the next
 *          persistent grouped launch (value < 0 disables), so that its
 *          consumers' bounded waits expire; the launch completes with
 *          invalid results and PE_ETIMEOUT is latched.
 *   key 2: wait limit of the persistent kernel in nanoseconds (0 = default).
 *   key 3: make the next workspace allocation fail (value != 0).
 *   key 4: device address of a buffer of 32 int64 per persistent CTA to
 *          which tcgen05 launches add per-role cycle counts (the caller
 *          zeroes it; 0 disables; while set, calls enqueue directly,
 *          without a graph).
 *   key 5: k-block (32 or 64) of tcgen05 plans built from now on (0 = default).
 *   key 6: tile order of tcgen05 plans built from now on (-1 = autotuned):
 *          0 phase-major longest-first, 1 phase-major column-grouped raster,
 *          2/3/4 lagged interleave of phases across matrices (lag 4/8/16).
 *   key 7: kernel mode of tcgen05 plans built from now on (-1 = autotuned,
 *          0 = one CTA per 128x256 tile, 2 = 2-SM UMMA on 256x256 tiles when
 *          every size is a multiple of 256, 3 = mode 2 with twelve epilogue
 *          warps and four operand stages instead of eight and five); any other
 *          value is PE_EINVAL.
 *   key 8: accumulators per CTA of 2-SM plans built from now on (1 or 2;
 *          0 = default).
 *   key 9: value != 0 turns off the pairing of BF16 matrices with a short
 *          side <= 64 in plans built from now on (0 = pairing on).
 * Returns PE_EINVAL for an unknown key.
 */
int pe_debug_set(int key, int64_t value);

/*
 * pe_polar_noalloc -- pe_polar on the plain FP32 path (PE_FP32) for one
 * matrix, for callers that must not have the library allocate device memory.
 * The paper has no counterpart; this is a deployment variant of the same
 * computation.
 *
 * Who needs it: programs whose own allocator takes all of device memory up
 * front (a framework's caching pool, an inference server with a fixed memory
 * budget), where an allocation by a library fails or fragments memory the
 * program has already accounted for; loops that cannot afford the
 * device-wide synchronisation that cudaMalloc and cudaFree can imply; hosts
 * that load this library as a plug-in that must allocate nothing.
 *
 * Workspace: a file-scope device array of 32 MiB inside the library, present
 * on every GPU where the library is loaded from load until process exit. The
 * call needs (2 s'L' + 2 s'^2) * 4 bytes plus a few KiB of descriptors, with
 * s' = min(m,n) and L' = max(m,n) rounded up to multiples of 128: e.g. every
 * GPT-2-small Muon matrix (768 x 3072 and smaller), or 1024 x 2048. Larger
 * matrices are rejected with PE_EINVAL and a message naming both sizes.
 * It calls no cudaMalloc, cudaFree or other allocating routine, and copies
 * nothing from host memory: a set-up kernel writes the descriptors.
 *
 * Sharing: all calls on a device use the same array, which keeps the last
 * call's contents; each call rewrites its descriptors and task lists and
 * clears what must start at zero. Calls whose work overlaps on the GPU
 * (different streams without ordering between them) race on the array and
 * give wrong results: issue them on one stream or order the streams.
 *
 * First call on a device: looks up the array's device address with
 * cudaGetSymbolAddress (which may load the module) and keeps it for the
 * process; make that first call before any stream capture. After
 * cudaDeviceReset the kept address is stale: this entry point does not
 * support a device reset.
 *
 *   X, m, n, table, T, stream  as for pe_polar (X: m x n row-major FP32, ld = n,
 *                              in/out, device memory).
 * Errors: PE_EINVAL (arguments, or the matrix does not fit the workspace),
 * PE_ECUDA. A non-finite input norm gives a non-finite output; there is no
 * status word for this entry point.
 */
int pe_polar_noalloc(void* X, int64_t m, int64_t n, const double* table, int T, void* stream);

/* --------------------------------------------------- fused Muon step
 *
 * The Muon update (Sec. 2.1): M <- beta M + (1 - beta) G,
 * W <- W - lr polar(M), with polar(M) by the Polar Express iteration of
 * pe_polar_batched. The momentum update is fused into the normalisation
 * kernel (it reads G and M once and writes M once) and the weight update into
 * the last polynomial step's epilogue (a TMA reduce-add of -lr X_T into W where
 * W's layout admits TMA, else a read-modify-write); polar(M) itself is never
 * stored.
 *   W, G, M  arrays of count device pointers to FP32 m[i] x n[i] row-major
 *            contiguous matrices: W in/out, G in, M in/out (M_0 = 0 is the
 *            caller's initialisation).
 *   beta     momentum coefficient in [0, 1] (paper default 0.9); the new M is
 *            fma(beta, M, (1 - beta) G) in FP32 with 1 - beta rounded to FP32.
 *   lr       learning rate; W(i, j) becomes W(i, j) + (-lr X_T(i, j)), the
 *            product and the sum each rounded to FP32.
 *   table, T, dtype, flags, stream  as for pe_polar_batched_ex (fixed
 *            normalisation constants 1.01 and 1e-7).
 * A plan is cached per (pointers, shapes, T, dtype, table, beta, lr); the
 * first call tunes it without changing M or W. Errors: as pe_polar_batched.
 */
int pe_muon_batched(void* const* W, void* const* G, void* const* M, const int64_t* m, const int64_t* n, int count,
                    double beta, double lr, const double* table, int T, int dtype, unsigned flags, void* stream);

/* ------------------------------------------------ long-side split (ranks)
 *
 * One matrix too large for one GPU, cut along its long side over R ranks
 * (the multi-device form of Alg. 1's online stage with A on the short side):
 * rank r holds G_r, the block of L_r of the L long-side columns (or rows) of
 * G, with the short side s shared. Then
 *   ||G||_F^2 = sum_r ||G_r||_F^2,   A = X X^T = sum_r X_r X_r^T,
 * B = b A + c A^2 is the same on every rank, and X_r <- a X_r + B X_r is
 * local: the iteration needs one all-reduce of a scalar before the first
 * step and one all-reduce of the s x s FP32 Gram per step, and nothing else.
 * The library computes every rank-local part; the caller performs the two
 * sums (e.g. NCCL all-reduce through torch.distributed) between the calls.
 *
 * Sequence on each rank, all on `stream`:
 *   pe_split_open -> pe_split_sumsq -> [sum over ranks] -> pe_split_set_norm
 *   -> for t = 0 .. T-1: pe_split_gram(t) -> [sum A over ranks] -> pe_split_step(t)
 *   -> pe_split_close.
 * pe_split_step(T - 1) writes the rank's block of the result into X.
 * With R = 1 the results are those of pe_polar_batched_ex with
 * PE_BATCH_PHASED | PE_BATCH_NO_GRAPH.
 */
typedef struct pe_split_s* pe_split_t;

/* X: the rank's block, rows x cols row-major (ld = cols), FP32, device
 * memory, in/out (read by pe_split_sumsq, overwritten by the last step).
 * short_is_rows = 1: the short side s = rows is shared and the ranks split
 * the columns (X_r = G_r); 0: s = cols is shared and the ranks split the
 * rows (X_r = G_r^T). Either local extent may be smaller than s.
 * table, T, dtype as for pe_polar (PE_FP32 or PE_BF16). The handle owns its
 * workspace until pe_split_close. Errors: PE_EINVAL, PE_ENOMEM, PE_ECUDA,
 * PE_EUNSUPPORTED (PE_BF16X3). */
int pe_split_open(void* X, int64_t rows, int64_t cols, int short_is_rows, const double* table, int T,
                  int dtype, void* stream, pe_split_t* handle);

/* Prepares the rank's block (cast, orientation, padding) and returns its
 * squared Frobenius norm in *sumsq (FP64, summed in a fixed order). Waits
 * for the stream. */
int pe_split_sumsq(pe_split_t handle, double* sumsq);

/* Sets the normalisation from the sum over ranks of pe_split_sumsq:
 * X_0 = G / (1.01 sqrt(total) + 1e-7) (Alg. 1; App. A constants). */
int pe_split_set_norm(pe_split_t handle, double total_sumsq);

/* The rank's partial Gram of step t (t = 0 .. T-1, in order), X_r X_r^T, as
 * a full symmetric s x s FP32 matrix into A (device memory, row-major,
 * leading dimension lda >= s). Step 0 includes the normalisation. */
int pe_split_gram(pe_split_t handle, int t, float* A, int64_t lda);

/* Step t given A = sum over ranks of the partial Grams (device memory, s x s
 * FP32, lda >= s): B = b_t A + c_t A^2, X_r <- a_t X_r + B X_r; the last step
 * writes X. */
int pe_split_step(pe_split_t handle, int t, const float* A, int64_t lda);

/* Frees the handle's workspace (after the stream's work has finished). */
int pe_split_close(pe_split_t handle);

/* ------------------------------------ fast rectangular iteration
 *
 * Alg. 4 (the appendix on fast polynomial iteration for rectangular
 * matrices) on the short side: with X the s x L normalised matrix, a block of
 * k polynomial steps takes Y = X X^T (plus shift * I in the first block only),
 * Q_0 = I, then per step R_t = Q_{t-1}^T Y Q_{t-1} and
 * Q_t = Q_{t-1} (a_t I + b_t R_t + c_t R_t^2), and finally X <- Q_k X: two
 * products with the long side per block instead of two per step. Steps run
 * in blocks of `restart` (the appendix's restarting strategy; restart = 1 is
 * the ordinary iteration up to the shift, restart >= T a single block).
 * The normalisation divides by 1.01 ||G||_F + norm_eps (the appendix
 * normalises by ||X||_F + 1e-3 with the shift).
 *
 * FP32 path only (dtype PE_FP32; other dtypes give PE_EUNSUPPORTED): the
 * s x s products are grouped SIMT FP32 GEMMs. Q tends to Y^{-1/2}, so FP32
 * rounding of Q reaches the result amplified by about the condition number of
 * the input's normalised spectrum.
 */

/* One matrix, in place: X as for pe_polar (FP32, row-major, ld = n, device),
 * table of T rows (a, b, c), restart in 1..64, shift = norm_eps = 1e-3 (the
 * appendix's values), no CUDA graph. Errors: as pe_polar. */
int pe_polar_fast(void* X, int64_t m, int64_t n, const double* table, int T, int restart, int dtype, void* stream);

/* A list of matrices in one grouped launch per product: X, m, n, count as
 * for pe_polar_batched; shift >= 0 added to Y in the first block; norm_eps
 * >= 0; flags PE_BATCH_* (graph capture as pe_polar_batched_ex). */
int pe_polar_fast_batched(void* const* X, const int64_t* m, const int64_t* n, int count, const double* table, int T,
                          int restart, double shift, double norm_eps, int dtype, unsigned flags, void* stream);

/* ------------------------------------ spectrum-aware initialisation
 *
 * For matrices with one dominant singular value (App. H, the case k = 1).
 * With X_0 = G / (1.01 ||G||_F + 1e-7) on the short side (as pe_polar
 * normalises) and f = ||X_0||_F: the power method (subspace iteration with
 * one vector) on X_0 X_0^T gives z <= sigma_1(X_0); the Frobenius identity
 * then bounds sigma_1 in [z, f] and every other singular value by
 * w = sqrt(f^2 - z^2). When the intervals [0, w] and [z, f] are disjoint
 * (2 z^2 > f^2, and z < f) the odd cubic p(x) = a x + b x^3 with
 * p(w) = p(z) = 1 (Eq. init_poly, as a polynomial of x / f) maps the spectrum
 * into [l', 1], l' = min(l / w, p(f)), and T Polar Express steps for [l', 1]
 * follow; otherwise T + 1 ordinary steps for [l, 1] (the cubic counts as a
 * step, as in the appendix's comparison).
 */

/* Lower bound of sigma_1 by `iters` power steps v <- X_0 X_0^T v / ||.||
 * from v0, then z = ||X_0^T v||.
 *   X      device, m x n row-major contiguous FP32 (ld = n); read only.
 *   v0     host, min(m, n) floats, nonzero and finite (the method's random
 *          start, drawn by the caller).
 *   iters  0..10000.
 *   z, f   host out: the bound z and f = ||X_0||_F (both 0 for G = 0).
 * Synchronises `stream` (the bound is needed on the host). Device buffers
 * are allocated and freed per call. Errors: PE_EINVAL, PE_ECUDA. */
int pe_spectrum_bound(const void* X, int64_t m, int64_t n, const float* v0, int iters, double* z, double* f,
                      void* stream);

/* Option of pe_spectrum_aware_table_ex / pe_polar_spectrum_aware_ex (not in
 * the appendix): keep the cubic only when the greedy lower bound (Thm. 1)
 * of its composition after the last step exceeds that of the plain
 * composition with T + 1 steps. */
#define PE_SPECTRUM_GATE 1u

/* Host: the coefficient table of the initialised iteration, T + 1 rows of
 * (a, b, c) into table (caller-owned, 3 (T + 1) doubles): row 0 the cubic
 * (a, b, 0) and rows 1..T the pe_coeffs(5, l', T, 1.01) composition, or, when
 * the cubic does not apply, pe_coeffs(5, l, T + 1, 1.01). z is used as given.
 * info (nullable, 6 doubles): applied (1 or 0), the z used, f, a, b, l'.
 * T in 0..63, l in (0, 1]. Errors: PE_EINVAL, PE_ENOCONV. */
int pe_spectrum_aware_table(double z, double f, double l, int T, double* table, double* info);

/* As pe_spectrum_aware_table, with z first shrunk to z (1 - z_safety),
 * z_safety in [0, 1) (a caller whose z carries rounding error keeps it below
 * sigma_1), and flags 0 or PE_SPECTRUM_GATE. */
int pe_spectrum_aware_table_ex(double z, double f, double l, int T, double z_safety, unsigned flags, double* table,
                               double* info);

/* pe_spectrum_bound, pe_spectrum_aware_table_ex, then pe_polar with that
 * table (T + 1 steps) on X in place. X as for pe_polar (FP32, device,
 * in/out); dtype PE_FP32, PE_BF16 or PE_BF16X3; z_safety and flags as for
 * pe_spectrum_aware_table_ex; info as for pe_spectrum_aware_table. Each call
 * builds a plan for its data-dependent table (a cached tuned schedule of the
 * same shape is reused). Errors: as the three calls. */
int pe_polar_spectrum_aware_ex(void* X, int64_t m, int64_t n, double l, int T, int dtype, const float* v0, int iters,
                               double z_safety, unsigned flags, double* info, void* stream);

/* pe_polar_spectrum_aware_ex with z_safety = 1e-5 (the bound z is computed
 * in FP32 on the GPU; the shrink keeps its rounding from lifting it above
 * sigma_1) and flags 0 (the appendix's rule). */
int pe_polar_spectrum_aware(void* X, int64_t m, int64_t n, double l, int T, int dtype, const float* v0, int iters,
                            double* info, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* POLAR_EXPRESS_H */
