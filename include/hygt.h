/*
 * hygt.h -- C ABI of libhygt.so, the GB300 (sm_103a) implementation of the
 * Hypercube-Givens Transform (HyGT) of Said et al., "Highly Efficient
 * Non-Separable Transforms for Next Generation Video Coding".
 *
 * Definitions (Sec. II-IV of the paper):
 *   - A block is a vector of N = 2^log2n residual values (Sec. II: the
 *     residual vector r; a 4x4 block is N = 16, an 8x8 block N = 64, a 16x16
 *     block N = 256), stored contiguously in raster order.
 *   - Each block carries a transform-set index (Sec. II: the classification
 *     index c, sent as side information; Sec. VI: 35 intra modes x 3
 *     candidates = 105 sets per block size, or no secondary transform).
 *     HYGT_SKIP_SET selects "no transform" (identity).
 *   - A set is R rounds (Sec. IV, Fig. 2).  Round r is log2n passes; pass p
 *     rotates every pair (m, n = m + 2^p), m with bit p clear, numbered
 *     j = 0..N/2-1 by increasing m (Sec. IV, Fig. 3 and Fig. 4), by its own
 *     angle theta[set][r][p][j] (R N log2(N) / 2 angles per set, Sec. IV):
 *     (a, b) -> (cos*a + sin*b, -sin*a + cos*b) (Givens matrix, Sec. IV).
 *   - After round r an optional permutation slot gathers v'[i] = v[perm[r][i]]
 *     (the optional sorting pass of Fig. 2, allowed after every round).
 *   - The inverse applies the passes in reverse order with negated angles
 *     and undoes each permutation (Sec. III inverse product; Sec. IV).
 *   - Integer path (Sec. IV, Fig. 5, "on-the-fly conversion" and the
 *     integer-arithmetic requirement): an angle index q of angle_bits bits
 *     stands for theta = 2*pi*q / 2^angle_bits and is converted to the
 *     multipliers c = round(2^f cos theta), s = round(2^f sin theta),
 *     f = frac_bits; every butterfly output is rounded half up,
 *     floor((c*a + s*b + 2^(f-1)) / 2^f), in int32.  The inverse uses (c, -s).
 *
 * Conventions:
 *   - Device pointers (prefix d_) are global-memory pointers on the current
 *     device, owned by the caller, 16-byte aligned; otherwise HYGT_ERR_ARG.
 *     Host pointers (prefix h_) are read during the call only.
 *   - Compute calls are asynchronous on `stream` (NULL = legacy default
 *     stream).  Argument errors are returned synchronously, before any
 *     launch; a launch failure returns HYGT_ERR_CUDA.
 *   - d_status (nullable) is a device int the caller zero-initialises.  A
 *     condition detected on the device (a set index >= num_sets that is not
 *     HYGT_SKIP_SET) writes its hygt_status code there (first error wins)
 *     and that block's output is all zeros.  Kernels never trap or abort.
 *   - A plan owns its device tables until hygt_destroy.  A plan may be used
 *     from several streams at once; it is never modified by compute calls.
 */
#ifndef HYGT_H
#define HYGT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

struct CUstream_st;
/* Same type as cudaStream_t. */
typedef struct CUstream_st *hygt_stream;

/* Opaque plan: one block size, one round count, num_sets parameter sets. */
typedef struct hygt_plan_s *hygt_plan;

typedef enum hygt_status {
  HYGT_OK = 0,
  HYGT_ERR_ARG = 1,         /* bad argument (shape, pointer, alignment, permutation) */
  HYGT_ERR_CUDA = 2,        /* a CUDA runtime call or launch failed */
  HYGT_ERR_OOM = 3,         /* device allocation failed */
  HYGT_ERR_SET_INDEX = 4,   /* device: set index >= num_sets and != HYGT_SKIP_SET */
  HYGT_ERR_UNSUPPORTED = 6, /* plan kind does not support this call */
  HYGT_ERR_TOO_LARGE = 7    /* batch larger than the static scratch of hygt_forward_static */
} hygt_status;

#define HYGT_SKIP_SET 0xFFFFu
#define HYGT_MAX_LOG2N 8
#define HYGT_MAX_ROUNDS 8

/*
 * Build a plan for the integer path (Sec. IV, Fig. 5) and the FP32 path on
 * the same angles.
 *   log2n       1..8 (N = 2..256).
 *   rounds      1..8.
 *   num_sets    1..65535.
 *   h_angle_idx host uint8 [num_sets][rounds][log2n][N/2]: angle indices q,
 *               each < 2^angle_bits (one byte per parameter, Sec. IV).
 *   h_perms     host uint16 [num_sets][rounds][N] gather permutations (slot r
 *               applied after round r), or NULL for none.  Each slot must be
 *               a permutation of 0..N-1.
 *   angle_bits  1..8.   frac_bits 1..10.
 * The FP32 path of this plan uses cos/sin of theta = 2*pi*q / 2^angle_bits,
 * evaluated in FP64 on the host and rounded to FP32.
 * Allocates the plan's device tables on the current device (synchronous).
 */
hygt_status hygt_create(hygt_plan *out, int log2n, int rounds, int num_sets,
                        const uint8_t *h_angle_idx, const uint16_t *h_perms,
                        int angle_bits, int frac_bits);

/*
 * Build a plan for the FP32 path with free angles (the parametrisation
 * optimised in Sec. V).  h_theta is host float [num_sets][rounds][log2n][N/2]
 * in radians; h_perms as for hygt_create.  Integer calls on such a plan
 * return HYGT_ERR_UNSUPPORTED.
 */
hygt_status hygt_create_float(hygt_plan *out, int log2n, int rounds, int num_sets,
                              const float *h_theta, const uint16_t *h_perms);

/* Release the plan's device tables (synchronises the device). NULL is a no-op. */
void hygt_destroy(hygt_plan plan);

/*
 * Integer forward HyGT (Sec. IV): d_x int16 [nblocks][N] -> d_y int32
 * [nblocks][N].  d_set: uint16 [nblocks] set indices, or NULL for set 0 on
 * every block.  A block with HYGT_SKIP_SET is copied (widened).
 * For every int16 input the int32 intermediates cannot overflow.
 */
hygt_status hygt_forward(hygt_plan plan, const int16_t *d_x, int32_t *d_y,
                         const uint16_t *d_set, int64_t nblocks, hygt_stream stream,
                         int *d_status);

/*
 * Integer inverse HyGT (Sec. III inverse product, Sec. IV negative angles):
 * d_y int32 [nblocks][N] -> d_x int16 [nblocks][N], saturated to
 * [-32768, 32767].  A block with HYGT_SKIP_SET is narrowed with saturation.
 * Precondition: each block's L2 norm is at most 2^21, which holds for every
 * output of hygt_forward on int16 input; beyond it int32 arithmetic may wrap
 * (the call still completes, without a fault).
 */
hygt_status hygt_inverse(hygt_plan plan, const int32_t *d_y, int16_t *d_x,
                         const uint16_t *d_set, int64_t nblocks, hygt_stream stream,
                         int *d_status);

/* FP32 forward / inverse HyGT: float [nblocks][N] -> float [nblocks][N]
   (no rounding between passes).  Set handling as for the integer calls. */
hygt_status hygt_forward_f32(hygt_plan plan, const float *d_x, float *d_y,
                             const uint16_t *d_set, int64_t nblocks, hygt_stream stream,
                             int *d_status);
hygt_status hygt_inverse_f32(hygt_plan plan, const float *d_y, float *d_x,
                             const uint16_t *d_set, int64_t nblocks, hygt_stream stream,
                             int *d_status);

/*
 * Set-bucketed batch path for the integer transform (same results as
 * hygt_forward / hygt_inverse, bit for bit).  The per-block set index is the
 * classification index of Sec. II; blocks are first bucketed by set so that
 * the blocks of each warp share their multipliers, then transformed.
 *
 *   hygt_batch_workspace_bytes  device bytes of the schedule for nblocks
 *                               blocks, with the 16 bytes of counters of
 *                               the dynamic tail at its end (0 if nblocks
 *                               is out of range).
 *   hygt_batch_build            buckets d_set (uint16 [nblocks]; NULL = set 0)
 *                               into the caller's workspace d_work (16-byte
 *                               aligned, >= the bytes above) and zeroes the
 *                               tail's counters, async on stream.
 *   hygt_forward_batch /        transform with a schedule built for the same
 *   hygt_inverse_batch          plan set count and nblocks (a schedule built
 *                               for other sizes makes the call write
 *                               HYGT_ERR_ARG to d_status and no output).  One
 *                               schedule serves any number of forward and
 *                               inverse calls while d_set is unchanged.
 * nblocks <= 2^30, every block size of hygt_create.  Skip and bad set
 * indices behave as in hygt_forward / hygt_inverse.
 */
size_t hygt_batch_workspace_bytes(hygt_plan plan, int64_t nblocks);
hygt_status hygt_batch_build(hygt_plan plan, const uint16_t *d_set, int64_t nblocks,
                             void *d_work, size_t work_bytes, hygt_stream stream);
hygt_status hygt_forward_batch(hygt_plan plan, const void *d_work, const int16_t *d_x,
                               int32_t *d_y, int64_t nblocks, hygt_stream stream,
                               int *d_status);
hygt_status hygt_inverse_batch(hygt_plan plan, const void *d_work, const int32_t *d_y,
                               int16_t *d_x, int64_t nblocks, hygt_stream stream,
                               int *d_status);

/*
 * Launch tuning of the set-bucketed kernels (no counterpart in the paper:
 * how many blocks a CTA holds and how far ahead the input is staged decide
 * how well a GB300 SM hides memory latency; the autotuner of the Python
 * package times the choices and sets the fastest).  Per plan and direction
 * (inverse 0: hygt_forward_batch, 1: hygt_inverse_batch), used by every
 * later bucketed call with that plan, the mixed calls included:
 *   warps_per_cta  warps of a CTA, 1 .. max_warps (0: max_warps); a warp
 *        task holds 32 * (blocks per lane group) / (lanes per block) blocks;
 *   ctas_per_sm    CTAs per SM, 1 .. 8 (0: as many as the shared memory and
 *        registers allow); the shared memory is split between them;
 *   stage          -1: the default; 0: blocks read straight from global
 *        memory; 1: each warp copies its next task's blocks into shared
 *        memory (cp.async) while it transforms the current one; 2: each
 *        warp prefetches its next task's blocks into L2; 3: as 1, by one
 *        bulk copy (cp.async.bulk, completing on a per-warp mbarrier) per
 *        block; an input that is not 16-byte aligned falls back to 0 (N >= 16
 *        for 1, 2 and 3; smaller blocks return HYGT_ERR_UNSUPPORTED).  A bulk
 *        copy that has not landed within about a second makes the warp stop
 *        and write HYGT_ERR_CUDA to d_status; 4: no staging, and the warp
 *        tasks taken in an order interleaved across the sets (task t of
 *        every set, then task t + 1, ..., the warps of all CTAs sweeping the
 *        sets together) instead of one contiguous range per warp, so that
 *        blocks sharing a 128-byte line, which belong to different sets, are
 *        read while the line is still in L2; with ctas_per_sm 0 as many CTAs
 *        as the registers allow, reading the set tables from global memory,
 *        else each CTA holds the tables of all sets in shared memory when
 *        they fit its share (4x4 blocks in layouts 0 and 2; other block sizes and
 *        layouts return HYGT_ERR_UNSUPPORTED; the single mixed launch runs
 *        such a class in its layout's first menu entry);
 *   layout         0: a block spread over a group of lanes (several values
 *        per lane, cross-lane passes by shuffles, several blocks per lane
 *        group sharing each multiplier load); 1: one lane per block (every
 *        pass in registers, multipliers shared by the warp's blocks through
 *        broadcast loads; 4x4 and 8x8 blocks); 2: more values per lane and
 *        fewer blocks per lane group (8x8, 16x16: 32 values, 2 blocks) or
 *        the reverse (4x4: 4 values, 8 / 4 blocks); 3: layout 0 with 8
 *        blocks per lane group in the inverse as in the forward (4x4, 8x8);
 *        4: layout 0 with the cross-lane passes done as register passes on
 *        the block transposed through shared memory (4x4, 8x8, 16x16); 5:
 *        layout 4 with 2 blocks per lane group (16x16).  Layouts 1 to 5
 *        take stage -1 .. 2 (layout 2 also 4 for 4x4 blocks); other block
 *        sizes, and stage 3, return HYGT_ERR_UNSUPPORTED.  The
 *        secondary-transform calls use layout 0 whatever is set, and run
 *        stage 4 as stage 0.
 * max_warps (get) is the largest warps_per_cta of the layout currently set.
 * Results do not depend on the tuning.  A choice whose shared memory does
 * not fit makes the next bucketed call return HYGT_ERR_UNSUPPORTED.  Not
 * thread-safe with concurrent calls on the same plan.
 */
hygt_status hygt_batch_set_tuning(hygt_plan plan, int inverse, int warps_per_cta,
                                  int ctas_per_sm, int stage, int layout);
hygt_status hygt_batch_get_tuning(hygt_plan plan, int inverse, int *warps_per_cta,
                                  int *ctas_per_sm, int *stage, int *layout, int *max_warps);

/*
 * Dynamic tail of the bucketed kernels (no counterpart in the paper; per plan
 * and direction, like the launch tuning).  The kernels give each warp one
 * contiguous range of the set-sorted order, fixed at launch; with a tail of
 * t / 64 (t = 1 .. 32; 0, the default, turns it off) the first (64 - t) / 64
 * of the order is split that way and the rest is handed out one warp task
 * at a time, through an atomic counter in the schedule workspace, to the
 * warps that finish their range, so that SMs done early take the work of
 * late ones.  The tail's tasks read their set tables from global memory and
 * run without a stage.  For 8x8 blocks in layouts 0 and 3 and 16x16 blocks
 * in layouts 0, 4 and 5, any stage but 4 (others return
 * HYGT_ERR_UNSUPPORTED, as does hygt_batch_set_tuning to such a point while
 * a tail is set).  Results do not depend on it.  The single mixed launch and
 * the secondary-transform calls do not use it.  One workspace serves one
 * call at a time: the last warp of a launch puts the counter back to zero.
 */
hygt_status hygt_batch_set_tail(hygt_plan plan, int inverse, int tail_64ths);
hygt_status hygt_batch_get_tail(hygt_plan plan, int inverse, int *tail_64ths);

/*
 * FP32 HyGT through the same set-bucketed schedule (the FP32 forward and
 * inverse of Sec. IV; y_m = c a + s b, y_n = -s a + c b in FP32, the inverse
 * with (c, -s) and the passes reversed): hygt_batch_build(plan, d_set, ...)
 * first, then these calls with the same d_work and nblocks (float
 * [nblocks][N] in and out, 16-byte aligned).  For N >= 16 (log2n >= 4;
 * smaller blocks return HYGT_ERR_UNSUPPORTED: use hygt_forward_f32).  Skip
 * blocks are copied; bad set indices give zeros and HYGT_ERR_SET_INDEX in
 * d_status; a schedule built for another batch gives HYGT_ERR_ARG in
 * d_status and no output.  Async on stream.
 */
hygt_status hygt_forward_batch_f32(hygt_plan plan, const void *d_work, const float *d_x,
                                   float *d_y, int64_t nblocks, hygt_stream stream,
                                   int *d_status);
hygt_status hygt_inverse_batch_f32(hygt_plan plan, const void *d_work, const float *d_y,
                                   float *d_x, int64_t nblocks, hygt_stream stream,
                                   int *d_status);

/*
 * Differentiable FP32 path (the angles are the parameters optimised in
 * Sec. V; the paper leaves the optimiser out of scope).
 *
 *   hygt_update_theta  recompute the (cos, sin) table of an FP32 plan from
 *        device angles d_theta (float [num_sets][rounds][log2n][N/2], radians),
 *        async on stream; order it with other calls that use the plan.
 *        Integer plans return HYGT_ERR_UNSUPPORTED.
 *   hygt_backward_workspace_bytes  device bytes hygt_backward_f32 needs for
 *        nblocks blocks (0 if the plan has too many angles: the shared-memory
 *        accumulators of one warp must fit in one CTA).
 *   hygt_backward_f32  given the forward output d_y and dL/dy d_gy (float
 *        [nblocks][N]), writes dL/dx to d_gx (float [nblocks][N]; must not
 *        alias d_y or d_gy) and dL/dtheta to d_gtheta (double, layout of the
 *        angles; overwritten).  For each rotation, dL/dtheta gets
 *        g_m y_n - g_n y_m (y = the rotation's outputs, g = their
 *        gradients); each pass's input is recomputed from its output by the
 *        inverse rotation, so nothing is stored between forward and
 *        backward.  The sum over blocks is deterministic (fixed order; FP32
 *        within a block slot, FP64 across slots and CTAs).  Skip blocks pass
 *        dL/dy through and add nothing; bad set indices give zero dL/dx and
 *        HYGT_ERR_SET_INDEX in d_status.
 */
hygt_status hygt_update_theta(hygt_plan plan, const float *d_theta, hygt_stream stream);
size_t hygt_backward_workspace_bytes(hygt_plan plan, int64_t nblocks);
hygt_status hygt_backward_f32(hygt_plan plan, const float *d_y, const float *d_gy, float *d_gx,
                              double *d_gtheta, const uint16_t *d_set, int64_t nblocks,
                              void *d_work, size_t work_bytes, hygt_stream stream,
                              int *d_status);

/*
 * The coding-gain objective of Sec. V and the angle fit it drives.
 *
 * Sec. V rates a transform T by the variance vector v = diag(T Phi T^T) of
 * its outputs (Phi the residuals' correlation matrix, Eq. 1) under the
 * high-rate model R(D) = 1/2 log2(eps^2 sigma^2 / D) of Sec. V; the paper's
 * optimiser searches the angles for the highest coding gain, with restarts,
 * and leaves its details out.  Here Phi is the correlation of a batch of
 * blocks, so v_i = (1/B) sum_b y_{b,i}^2 for the transformed batch y, and the
 * objective is the average rate per coefficient up to constants,
 *     J = 1/(2N) sum_i log2 v_i
 * (minimising J maximises the coding gain mean(v) / geomean(v); an
 * orthogonal T cannot go below the KLT's value, Eq. 2).
 *
 *   hygt_coding_gain_workspace_bytes  device bytes hygt_coding_gain_f32 needs
 *        (0 for N = 2, nblocks < 1 or a null plan).
 *   hygt_coding_gain_f32  from the FP32 outputs d_y (float [nblocks][N], one
 *        class: every block counts) writes v to d_v (double [N]), J to d_J
 *        (one double) and the weights w_i = 1 / (N ln 2 B v_i) to d_w
 *        (float [N]), for which dJ/dy_{b,i} = w_i y_{b,i}.  A coefficient
 *        with v_i = 0 gets w_i = 0 and makes J = -inf.  The sums are
 *        deterministic (fixed order; FP32 over runs of 8 values, FP64
 *        beyond).  Async on stream; the plan gives N only.
 *   hygt_backward_diag_f32  the backward of any loss whose gradient with
 *        respect to the outputs is diagonal, dL/dy_{b,i} = d_w[i] y_{b,i}
 *        (the coding-gain objective with w from hygt_coding_gain_f32; the
 *        energy-compaction loss (1/B) sum_{i>=K} y_i^2 with w_i = 2/B for
 *        i >= K): the same kernel as hygt_backward_f32, which forms dL/dy in
 *        registers instead of reading it.  d_gx (float [nblocks][N]) may be
 *        null, and then dL/dx is not written: the call reads d_y alone.
 *        Same workspace as hygt_backward_f32.
 *   hygt_adam_step  one Adam step (Kingma and Ba) on n FP32 parameters
 *        d_theta from the FP64 gradient d_grad, with FP32 moment buffers d_m
 *        and d_v (zero before step 1); step counts from 1.  The paper names
 *        no optimiser; this is the one the fit uses.
 */
size_t hygt_coding_gain_workspace_bytes(hygt_plan plan, int64_t nblocks);
hygt_status hygt_coding_gain_f32(hygt_plan plan, const float *d_y, int64_t nblocks, double *d_v,
                                 float *d_w, double *d_J, void *d_work, size_t work_bytes,
                                 hygt_stream stream);
hygt_status hygt_backward_diag_f32(hygt_plan plan, const float *d_y, const float *d_w,
                                   float *d_gx, double *d_gtheta, const uint16_t *d_set,
                                   int64_t nblocks, void *d_work, size_t work_bytes,
                                   hygt_stream stream, int *d_status);
hygt_status hygt_adam_step(float *d_theta, const double *d_grad, float *d_m, float *d_v,
                           int64_t n, float lr, float beta1, float beta2, float eps, int step,
                           hygt_stream stream);

/*
 * Secondary-transform pipeline (Sec. VI): the HyGT used as a secondary
 * transform on the low-frequency coefficients of a separable primary
 * transform -- a 4x4 HyGT (N = 16) for 4x4 blocks, an 8x8 HyGT (N = 64) on
 * the top-left 8x8 coefficients of 8x8, 16x16 and 32x32 blocks -- fused
 * with the primary in one kernel.  The paper does not fix the primary; it
 * is the orthonormal 2-D DCT-II in integer arithmetic with the HyGT's
 * precision: C = round(256 D), D[k][i] = a_k cos(pi (2i + 1) k / (2M)),
 * a_0 = sqrt(1/M), a_k = sqrt(2/M); each 1-D stage rounds half up,
 * floor((sum_i C[k][i] x_i + 128) / 256), rows then columns (the inverse:
 * C^T, columns then rows, then int16 saturation).  The sub-block is the
 * HyGT's vector in raster order (row-major); the other coefficients pass
 * through.
 *
 *   hygt_secondary_forward  int16 residual blocks d_x [nblocks][M*M]
 *        (raster, M = 2^log2m, log2m 2..5) -> int32 coefficients d_y
 *        [nblocks][M*M].  plan: an integer plan with log2n = 4 for
 *        log2m = 2 and log2n = 6 otherwise (else HYGT_ERR_ARG).  d_set as
 *        for hygt_forward: 0xFFFF = no secondary transform (primary only);
 *        other indices >= num_sets zero the block and write
 *        HYGT_ERR_SET_INDEX to d_status.  Pointers 16-byte aligned; async
 *        on stream.  Exact in int32 for every int16 input.
 *   hygt_secondary_inverse  int32 coefficients -> int16 blocks (inverse HyGT
 *        on the sub-block, then the inverse DCT-II); coefficients as the
 *        forward produces them keep every sum within int32.
 */
hygt_status hygt_secondary_forward(hygt_plan plan, int log2m, const int16_t *d_x, int32_t *d_y,
                                   const uint16_t *d_set, int64_t nblocks, hygt_stream stream,
                                   int *d_status);
hygt_status hygt_secondary_inverse(hygt_plan plan, int log2m, const int32_t *d_y, int16_t *d_x,
                                   const uint16_t *d_set, int64_t nblocks, hygt_stream stream,
                                   int *d_status);
/*
 *   hygt_secondary_forward_batch / hygt_secondary_inverse_batch  the same
 *        pipeline for 4x4 (log2m = 2) and 8x8 (log2m = 3) blocks, where the
 *        secondary covers every coefficient, through the set-bucketed
 *        kernels with the primary fused: hygt_batch_build(plan, d_set, ...)
 *        first, then these calls with its d_work and nblocks (same results,
 *        bit for bit; other log2m: HYGT_ERR_UNSUPPORTED).  The launch tuning
 *        of hygt_batch_set_tuning applies.
 */
hygt_status hygt_secondary_forward_batch(hygt_plan plan, const void *d_work, int log2m,
                                         const int16_t *d_x, int32_t *d_y, int64_t nblocks,
                                         hygt_stream stream, int *d_status);
hygt_status hygt_secondary_inverse_batch(hygt_plan plan, const void *d_work, int log2m,
                                         const int32_t *d_y, int16_t *d_x, int64_t nblocks,
                                         hygt_stream stream, int *d_status);

/*
 * General PMPT with explicit index vectors (Sec. III, Eq. 5; Sec. IV,
 * Eq. 7-9).  Each pass of each set is a parallel-Givens matrix over an
 * arbitrary cover of 0..N-1 by N/2 disjoint pairs (m_j, n_j) with one angle
 * per pair -- the construction the HyGT specialises by taking the pairs
 * from the hypercube, which saves the index storage.  The forward applies
 * pass 0 first; the inverse runs the passes in reverse with negated angles.
 * Rotation of a pair: y_m = c a + s b, y_n = -s a + c b; integer plans
 * round every output half up, floor((. + 2^(f-1)) / 2^f), in int32, and
 * the inverse saturates to int16.
 *
 *   hygt_pmpt_create  n even, 2..256; passes 1..4096; num_sets 1..65535;
 *        m_idx, n_idx host uint16 [num_sets][passes][n/2], every pass a cover
 *        of 0..n-1 (each index exactly once), else HYGT_ERR_ARG.  Exactly one
 *        of angle_idx (host uint8, same layout: theta = 2 pi q / 2^angle_bits,
 *        integer and FP32 calls) and theta (host float radians: FP32 calls
 *        only) is non-null.  Synchronous; allocates the plan's device tables
 *        on the current device.
 *   hygt_pmpt_forward / hygt_pmpt_inverse  integer (int16 -> int32 /
 *        int32 -> int16 saturated), d_* device [nblocks][n], 4-byte aligned;
 *        d_set (uint16 [nblocks] or null: set 0), 0xFFFF = identity, other
 *        indices >= num_sets zero the block and write HYGT_ERR_SET_INDEX to
 *        d_status (nullable, first error wins).  Async on stream.
 *   hygt_pmpt_forward_f32 / hygt_pmpt_inverse_f32  the same in FP32.
 *   hygt_pmpt_param_bytes  memory of the parameters at one byte per angle
 *        and one byte per index: 3 bytes per pair (the HyGT needs 1).
 */
typedef struct hygt_pmpt_s *hygt_pmpt;
hygt_status hygt_pmpt_create(hygt_pmpt *out, int n, int passes, int num_sets,
                             const uint8_t *angle_idx, const float *theta,
                             const uint16_t *m_idx, const uint16_t *n_idx, int angle_bits,
                             int frac_bits);
void hygt_pmpt_destroy(hygt_pmpt pmpt);
size_t hygt_pmpt_param_bytes(int n, int passes, int num_sets);
hygt_status hygt_pmpt_forward(hygt_pmpt pmpt, const int16_t *d_x, int32_t *d_y,
                              const uint16_t *d_set, int64_t nblocks, hygt_stream stream,
                              int *d_status);
hygt_status hygt_pmpt_inverse(hygt_pmpt pmpt, const int32_t *d_y, int16_t *d_x,
                              const uint16_t *d_set, int64_t nblocks, hygt_stream stream,
                              int *d_status);
hygt_status hygt_pmpt_forward_f32(hygt_pmpt pmpt, const float *d_x, float *d_y,
                                  const uint16_t *d_set, int64_t nblocks, hygt_stream stream,
                                  int *d_status);
hygt_status hygt_pmpt_inverse_f32(hygt_pmpt pmpt, const float *d_y, float *d_x,
                                  const uint16_t *d_set, int64_t nblocks, hygt_stream stream,
                                  int *d_status);

/*
 * Mixed block sizes in one persistent launch.  The paper's codec applies
 * 4x4 (N = 16) and 8x8 (N = 64) secondary transforms (Sec. VI); a frame
 * tiled into 4x4, 8x8 and 16x16 blocks gives one batch per block size, each
 * with its own plan, set indices and schedule.  One launch transforms all of
 * them, in one of three ways, chosen by the classes' `ctas`:
 *   - `ctas` > 0 for every class, summing to at most 4 * hygt_mixed_ctas():
 *     one launch; class c runs on its own `ctas` CTAs, concurrently with
 *     the others;
 *   - `ctas` = -1 for every class: one batch launch per class, one after
 *     the other on the stream (hygt_forward_batch's kernels);
 *   - otherwise (e.g. all 0): one launch; every CTA works through the
 *     classes in turn, each class spread over all CTAs.
 * A single launch sizes its shared memory for its largest class, which
 * leaves less L1 cache to the smaller ones; the autotuner of the Python
 * package times the three and keeps the fastest.  A single launch runs
 * each class in the staging and register layout of its plan's launch
 * tuning for that direction (hygt_batch_set_tuning) where its kernel has
 * that pair, from a short menu per block size:
 *   4x4    layout 0 (stage 0), layout 2 (stage 0 or 1);
 *   8x8    layout 0 (stage 1), layout 3 (stage 0 or 2);
 *   16x16  layout 0 (stage 0), layout 5 (stage 0 or 1), layout 4 (stage 0);
 * a tuning whose pair is not on the menu runs the first entry of its
 * layout, else layout 0 (stage -1 reads as the layout's default).  Warps
 * per CTA and CTAs per SM are the launch's own: one CTA per SM.
 *
 * Each class: plan = integer plan with N = 16, 64 or 256 (others return
 * HYGT_ERR_UNSUPPORTED; at most one class per block size, else
 * HYGT_ERR_ARG); d_set, nblocks, d_work / work_bytes as for
 * hygt_batch_build; d_x int16 [nblocks][N] forward input, d_y int32
 * [nblocks][N] coefficients (forward output, inverse input), d_xr int16
 * [nblocks][N] inverse output.  Data pointers 16-byte aligned.
 *
 *   hygt_forward_mixed / hygt_inverse_mixed  one launch over all classes,
 *        async on stream, with schedules already built (hygt_batch_build).
 *   hygt_mixed_graph_create  captures one whole step -- the schedules of
 *        all classes, the mixed forward, the mixed inverse -- into a CUDA
 *        graph (on private streams: the schedules are built on parallel
 *        branches that join before the forward; pointers and sizes are
 *        fixed at capture).  hygt_graph_launch replays it on `stream`;
 *        hygt_graph_destroy frees it.
 *   hygt_mixed_ctas  CTAs of one mixed launch on the current device.
 *   hygt_mixed_class_variant  the staging and register layout in which a
 *        single mixed launch runs a class of `plan` in direction `inverse`
 *        (0 forward, 1 inverse) under the plan's current tuning; stage and
 *        layout may be NULL.  HYGT_ERR_ARG for a NULL plan,
 *        HYGT_ERR_UNSUPPORTED for a floating-point plan or another N.
 */
typedef struct hygt_mixed_class {
  hygt_plan plan;
  const uint16_t *d_set;
  int64_t nblocks;
  void *d_work;
  size_t work_bytes;
  const int16_t *d_x;
  int32_t *d_y;
  int16_t *d_xr;
  int ctas;
} hygt_mixed_class;

typedef struct hygt_graph_s *hygt_graph;

int hygt_mixed_ctas(void);
hygt_status hygt_mixed_class_variant(hygt_plan plan, int inverse, int *stage, int *layout);
hygt_status hygt_forward_mixed(const hygt_mixed_class *classes, int nclasses,
                               hygt_stream stream, int *d_status);
hygt_status hygt_inverse_mixed(const hygt_mixed_class *classes, int nclasses,
                               hygt_stream stream, int *d_status);
hygt_status hygt_mixed_graph_create(hygt_graph *out, const hygt_mixed_class *classes,
                                    int nclasses, int *d_status);
hygt_status hygt_graph_launch(hygt_graph graph, hygt_stream stream);
void hygt_graph_destroy(hygt_graph graph);

/*
 * Dense matrix transform, the baseline of the comparison: y_b = K_{set(b)} x_b
 * with one N x N matrix per set (the matrix transform of Eq. 3; a KLT of
 * Eq. 2 is such a matrix).  Blocks are bucketed by set in tiles of 128.
 *
 *   dense_klt_create  h_K host float [num_sets][N][N], row-major (y = K x);
 *        N = 16, 64 or 256; builds BF16 and E4M3 operand images (N = 64,
 *        256; the E4M3 image of a set is K * 448 / max|K|) and the integer
 *        matrices round(2^frac_bits K) (|entries| <= 32767, else
 *        HYGT_ERR_ARG).  Synchronous.
 *   dense_klt_workspace_bytes / dense_klt_build  schedule of nblocks blocks
 *        (as hygt_batch_build), async on stream.
 *   dense_klt_apply  kind DENSE_KLT_BF16: BF16 x BF16 products with FP32
 *        accumulation on the tensor cores (tcgen05), d_y float [nblocks][N],
 *        N = 64 or 256; kind DENSE_KLT_FP8: E4M3 x E4M3 products with FP32
 *        accumulation on the tensor cores, each block scaled by 448 /
 *        max|x| (FP32) before rounding to E4M3 (saturating), the result
 *        scaled back by the block's and the set's scales, d_y float
 *        [nblocks][N], N = 64 or 256; kind DENSE_KLT_INT: d_y int32
 *        [nblocks][N] = floor((round(2^f K) x + 2^(f-1)) / 2^f) on the CUDA
 *        cores, N = 16 or 64.  Skip blocks are copied, bad set indices give
 *        zeros and HYGT_ERR_SET_INDEX in d_status.
 */
typedef struct dense_klt_s *dense_klt;
#define DENSE_KLT_BF16 0
#define DENSE_KLT_INT 1
#define DENSE_KLT_FP8 2
hygt_status dense_klt_create(dense_klt *out, int log2n, int num_sets, const float *h_K,
                             int frac_bits);
void dense_klt_destroy(dense_klt d);
size_t dense_klt_workspace_bytes(dense_klt d, int64_t nblocks);
hygt_status dense_klt_build(dense_klt d, const uint16_t *d_set, int64_t nblocks, void *d_work,
                            size_t work_bytes, hygt_stream stream);
hygt_status dense_klt_apply(dense_klt d, const void *d_work, const int16_t *d_x, void *d_y,
                            int64_t nblocks, int kind, hygt_stream stream, int *d_status);

/*
 * Bucketing plus integer forward transform with no device allocation.  The
 * paper has no counterpart: this is a calling convention of this library.
 *
 * Some callers cannot allocate device memory when they transform -- code
 * that runs where cudaMalloc is not allowed or not wanted (a real-time
 * encode loop, a host process that owns no device allocator, a library
 * layered under another runtime) -- so they cannot provide the workspace
 * that hygt_batch_build needs.  hygt_forward_static does the same work as
 * hygt_batch_build followed by hygt_forward_batch (same results, bit for
 * bit), with the schedule in a fixed 8 MiB array that the library holds in
 * the global memory of every GPU that loads it, until the process exits.
 *
 *   - The caller passes the plan (created beforehand), d_x, d_y, d_set and
 *     d_status exactly as for hygt_forward.
 *   - nblocks must satisfy hygt_batch_workspace_bytes(plan, nblocks) <=
 *     8,388,608 (about 2 million 8x8 blocks for 105 sets); larger batches
 *     return HYGT_ERR_TOO_LARGE before anything is launched.
 *   - The call allocates nothing itself.  Every call looks up the address
 *     of the current device's array (cudaGetSymbolAddress, a host-side
 *     query), so the call stays valid after a device reset.  The 8 MiB
 *     array is placed in device memory when the library's device code is
 *     loaded on that device; under CUDA's default lazy loading that is the
 *     first call of this function there, which can then fail with
 *     HYGT_ERR_CUDA when device memory is short.  Make one warm-up call at
 *     start-up (nblocks = 1 is enough), and make it before any stream
 *     capture.
 *   - All calls share the array and it keeps the last call's schedule; each
 *     call rebuilds the parts that must start at zero.  Calls whose work
 *     overlaps on the GPU (other streams, other host threads) race on the
 *     array: order them.
 */
hygt_status hygt_forward_static(hygt_plan plan, const int16_t *d_x, int32_t *d_y,
                                const uint16_t *d_set, int64_t nblocks, hygt_stream stream,
                                int *d_status);

/*
 * Host-buffer round trip of an integer batch: the forward transform of the
 * blocks in host memory, their coefficients, and the inverse transform
 * (reconstruction), all returned to host memory.  The paper's transform is
 * what runs (bucketing + hygt_forward_batch + hygt_inverse_batch); the pipe
 * adds the transfers: the batch goes through the GPU in chunks of
 * chunk_blocks blocks on three streams, so the host-to-device copy of one
 * chunk, the kernels of another and the device-to-host copies of a third
 * overlap.  Host buffers should be page-locked (cudaHostAlloc or
 * cudaHostRegister) for the copies to overlap; pageable memory works but
 * serialises them.
 *
 *   hygt_host_pipe_create  allocates, on the current device, three chunk
 *        slots (input, set indices, coefficients, reconstruction,
 *        schedule workspace, a stream and a status word each); chunk_blocks
 *        in 1 .. 2^26.  Synchronous.
 *   hygt_host_roundtrip    h_x int16 [nblocks][N] in; h_set uint16 [nblocks]
 *        or NULL (set 0); h_y int32 [nblocks][N] (or NULL: the coefficients
 *        are not copied back, only the reconstruction) and h_xr int16
 *        [nblocks][N] out.  Synchronous: returns when every result is in host memory;
 *        *h_status (nullable) receives the first device-side status
 *        (HYGT_ERR_SET_INDEX for an out-of-range set index).  Calls on one
 *        pipe must not overlap.
 *   hygt_host_pipe_destroy frees the slots (waits for them first).
 */
typedef struct hygt_host_pipe_s *hygt_host_pipe;
hygt_status hygt_host_pipe_create(hygt_host_pipe *out, hygt_plan plan, int64_t chunk_blocks);
hygt_status hygt_host_roundtrip(hygt_host_pipe pipe, const int16_t *h_x, const uint16_t *h_set,
                                int32_t *h_y, int16_t *h_xr, int64_t nblocks, int *h_status);
void hygt_host_pipe_destroy(hygt_host_pipe pipe);

/* Plan shape: any out-pointer may be NULL. */
hygt_status hygt_plan_info(hygt_plan plan, int *log2n, int *rounds, int *num_sets,
                           int *is_float);

/*
 * Bytes of transform parameters at one byte per angle (Sec. IV: R N log2(N)/2
 * angles per set; "one byte per parameter"), for num_sets sets.
 * Returns 0 for out-of-range arguments.  Host only.
 */
size_t hygt_param_bytes(int log2n, int rounds, int num_sets);

/* Static English text for a status code. */
const char *hygt_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* HYGT_H */
