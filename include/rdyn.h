/*
 * rdyn.h -- batched serial-chain dynamics on one GB300 GPU (sm_103a).
 *
 * C ABI of librdyn.so. No C++ or PyTorch types cross it: host arrays are
 * plain double pointers, batch arrays are raw device pointers, and the CUDA
 * stream is passed as an opaque pointer (a cudaStream_t; NULL = the legacy
 * default stream).
 *
 * Method: "Parallel Dynamics Computation using Prefix Sum Operations"
 * (Yang, Wu, Pan; arXiv 1609.04493). Inverse dynamics is the recursive
 * Newton-Euler algorithm (Sec. II-A, Eqs. id-forward and id-backward), cast
 * as a forward scan over SE(3) x se(3)^2 (Sec. III-B, Eq. scan-id-vel-acc)
 * and a backward scan of reaction wrenches (Sec. III-C, Eq. id-bkwd-scan).
 *
 * Conventions shared by every entry point:
 *   - twists are (v, w), linear part first; wrenches are (f, n), paired
 *     with twists as F^T V;
 *   - f_{i-1,i} = M_i exp([S_i] q_i) maps frame-i coordinates to frame i-1;
 *     M_i is its value at q_i = 0 and S_i is expressed in frame i;
 *   - the base frame is frame 0; V_0 and dV_0 are expressed in it; gravity
 *     enters as a base acceleration (dV_0 = (0, 0, 9.81, 0, 0, 0) for
 *     gravity along -z);
 *   - F_{n+1} is the wrench that link n exerts on its environment,
 *     expressed in frame n.
 *
 * Error behaviour: every int-returning call returns RD_OK (0) on success or
 * a negative RD_ERR_* code; rd_last_error() then gives a message for the
 * calling thread. Calls that take a stream are asynchronous with respect to
 * the host: an error detected on the host is returned at once, a launch
 * failure is returned as RD_ERR_CUDA, and faults inside a kernel surface on
 * the stream as usual CUDA errors.
 */
#ifndef RDYN_H
#define RDYN_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Opaque handle to a robot model resident on one device. */
typedef struct rd_model rd_model;

enum rd_dtype { RD_F32 = 0, RD_F64 = 1 };

enum rd_status {
    RD_OK = 0,
    RD_ERR_ARG = -1,     /* null pointer, bad size, invalid model data */
    RD_ERR_DTYPE = -2,   /* dtype not RD_F32 / RD_F64 */
    RD_ERR_RANGE = -3,   /* n outside [1, RD_MAX_LINKS] or B negative */
    RD_ERR_CUDA = -4,    /* a CUDA runtime call failed */
    RD_ERR_TIMEOUT = -5, /* a bounded device wait ran out */
    RD_ERR_ALLOC = -6    /* host or device allocation failed (create only) */
};

/* aba_batch flag: run the z_hat / lambda recursions in the data precision
 * (FP32 for RD_F32) instead of the precision of the articulated-inertia update
 * (FP64 or double-float), which the update and the Omega solves keep. */
#define RD_ABA_SCANS_IN_DTYPE 0x1
/* aba_batch flag: run the joint-frame kernel (full 6x6 congruence, FP64 update)
 * instead of the common-normal ones, for comparisons. */
#define RD_ABA_JOINT_FRAMES 0x2
/* aba_batch flag, RD_F32 only. By default the articulated-inertia update, the
 * Omega solves and the z_hat / lambda recursions of FP32 data run in
 * double-float arithmetic (a value is the unevaluated sum of two FP32 numbers,
 * about 48 significand bits; Dekker 1971) on the FP32 pipe, in common-normal
 * frames (constants as a kernel parameter for n % 4 == 0, n <= 64 and aligned
 * rows; in global memory otherwise). This flag runs them in hardware FP64
 * instead, in the same frames. Ignored for RD_F64. */
#define RD_ABA_FP64_UPDATE 0x4

/* aba_batch flags, RD_F32 only: the precision of the bias sweeps (the motion and
 * bias wrenches of tau_bias = ID(q, qd, 0, ...), the wrench carry, tau_hat and
 * the joint sin/cos). Along a long chain under gravity the bias torques grow
 * far above tau, and their FP32 rounding, amplified by the conditioning of
 * M(q), sets the error of qdd (n = 128: 2e-3 of max|qdd|). By default chains
 * longer than RD_ABA_EXTENDED_BIAS_LINKS run these sweeps in double-float
 * arithmetic (about 48 bits, on the FP32 pipe), shorter ones in FP32.
 * RD_ABA_EXTENDED_BIAS asks for double-float at any n, RD_ABA_FP32_BIAS for
 * FP32 at any n (comparisons). Ignored for RD_F64, whose sweeps run in FP64. */
#define RD_ABA_EXTENDED_BIAS 0x8
#define RD_ABA_FP32_BIAS 0x10
#define RD_ABA_EXTENDED_BIAS_LINKS 64
/* aba_batch flags: the mapping of instances to threads. One thread per
 * instance runs the three sweeps of the recursion serially; one warp per
 * instance (Sec. III-D) runs tau_bias by the scans of inverse dynamics across
 * its lanes, the articulated-inertia recursion (Eq. abi) link by link with each
 * link's update spread over 21 lanes, and the z_hat / c_hat and lambda / qdd
 * recursions (Eqs. fd-bkwd-scan, fd-fwd-scan) as scans across its lanes. The
 * warp mapping suits batches too small to fill the GPU with threads. Without
 * either flag the library picks by the batch size and n. Not combinable with
 * RD_ABA_JOINT_FRAMES or RD_ABA_SCANS_IN_DTYPE. */
#define RD_ABA_WARP_PER_INSTANCE 0x20
#define RD_ABA_THREAD_PER_INSTANCE 0x40
/* aba_batch flag: two warps per 32 instances, one running the
 * articulated-inertia recursion (Eq. abi, which depends on q only) and the other
 * the bias sweeps, tau_hat, z_hat and c_hat beside it, then lambda and qdd
 * (global constants, any n). Not combinable with the other mapping flags,
 * RD_ABA_JOINT_FRAMES or RD_ABA_SCANS_IN_DTYPE. */
#define RD_ABA_TWO_WARPS 0x80
/* aba_batch flag: as RD_ABA_TWO_WARPS with the articulated-inertia recursion
 * itself split over two warps by block of the 6x6 inertia (one the
 * translational and rotational diagonal blocks, the other the off-diagonal
 * block, exchanging their shift terms per link), three warps per 32 instances.
 * Same results to rounding; same exclusions. */
#define RD_ABA_THREE_WARPS 0x100
/* aba_batch test hook, only with RD_ABA_TWO_WARPS: the articulated-inertia warp
 * withholds its per-link announcements, so every wait of the other warp runs
 * out (one bounded wait per instance, a quarter of a second or more) and every
 * status word carries RD_WARN_TIMEOUT. qdd is then undefined. It exists to
 * test that path: no wait in the library is unbounded. */
#define RD_ABA_TEST_WITHHOLD 0x40000000

/* Per-instance status word of aba_batch (0 = fine); bits. */
#define RD_WARN_SINGULAR 1 /* an Omega_i <= 0 or a non-finite qdd appeared */
#define RD_WARN_TIMEOUT 2  /* two- or three-warp mapping (also fleets' warp pairs): a
                              bounded wait for another warp gave up (a quarter of a
                              second or more); that instance's qdd is invalid */

/* Kernel variant for rnea_batch. */
enum rd_variant {
    RD_VARIANT_AUTO = 0,    /* library's choice for (n, B, dtype) */
    RD_VARIANT_SERIAL = 1,  /* one thread per instance, per-link state in shared memory */
    RD_VARIANT_SERIAL_RECOMPUTE = 2, /* one thread per instance, backward sweep re-derives
                                        V_{i-1}, dV_{i-1} from V_i, dV_i; no per-link state */
    RD_VARIANT_SERIAL_RECOMPUTE_CS = 3, /* as 2, keeping cos/sin of q_i in shared memory */
    RD_VARIANT_SERIAL_REGSTATE = 4, /* as 1, the state of the first links (RD_TUNE_REGLINKS,
                                       default 16) held in registers, the rest in shared memory;
                                       needs n % 4 == 0 and 16-byte aligned rows */
    RD_VARIANT_SERIAL_HYBRID = 5, /* one thread per instance, per-link state in shared memory
                                    for the first K links only (RD_TUNE_STORED_LINKS(K), K a
                                    multiple of 4; 0 = library default); the backward sweep
                                    re-derives the motion of links K..n-1 as variant 2 does */
    RD_VARIANT_SERIAL_DH = 6, /* one thread per instance in common-normal link frames: each
                                 link transform is Rx(alpha_i) Rz(theta0_i + q_i) plus an offset
                                 (the Denavit-Hartenberg structure), built once by
                                 rd_model_create. With n % 4 == 0, n <= 128 and 16-byte aligned
                                 rows the link constants travel as a kernel parameter and the
                                 full backward-sweep state is kept for the first K links
                                 (RD_TUNE_STORED_LINKS(K); 0 = library default), cos/sin only
                                 for the rest, whose motion is re-derived; otherwise every link
                                 keeps its state in shared memory. AUTO takes this kernel for
                                 FP32 batches of more than 2048 whole-chunk rows. */
    RD_VARIANT_SERIAL_DH_RECOMPUTE = 7, /* as 6 with K = 0 (no full state) */
    RD_VARIANT_SERIAL_DH_TMEM = 8, /* as 6 (FP32, n <= 32, n % 4 == 0, aligned rows) with the
                                      state of the first 16 links in tensor memory: blocks of
                                      128 threads, four per SM, each owning 128 TMEM columns;
                                      K by RD_TUNE_STORED_LINKS (0 = largest that fits) */
    RD_VARIANT_SERIAL_DF = 9 /* RD_F64 data only, n <= 64, rows of any alignment: one thread
                                per instance in common-normal frames with every value a
                                double-float pair (two FP32 numbers, about 48 significand
                                bits; Dekker 1971) on the FP32 pipe instead of FP64; cos/sin
                                of q_i (sin/cos by Cody-Waite reduction and Taylor series,
                                see rd_joint_trig_df) kept in shared memory, motion
                                re-derived in the backward sweep. Relative error a few units
                                of 2^-48 per operation, for values within the FP32 exponent
                                range (magnitudes about 1e-38 to 3e38). Never chosen by
                                AUTO. */
};
/* Lane-parallel scan: L lanes of one warp per instance, L in {2,4,8,16,32};
 * each lane owns ceil(n/L) consecutive links, lanes combine their segments
 * with warp-shuffle log-step semigroup scans (Sec. III). */
#define RD_VARIANT_SCAN(L) (0x100 | (L))
/* OR-able flag: in FP32, evaluate sin/cos of q_i by a 2*pi range reduction
 * plus the special-function-unit approximation (absolute error ~4e-7) instead
 * of the default: the library routine in the joint-frame kernels, an FMA-pipe
 * polynomial (absolute error < 1.2e-7, see rd_joint_trig) in the
 * common-normal-frame kernels. Faster; the torque error can then exceed 1e-4
 * of max|tau| on instances whose torques nearly cancel. */
#define RD_FLAG_FAST_TRIG 0x1000
/* OR-able flag for rnea_batch_host: stage the arrays through device buffers
 * with the copy engines even where the kernel could read them in place. */
#define RD_FLAG_HOST_COPY 0x4000
/* OR-able tuning field: threads per block of the one-thread-per-instance
 * kernels (32, 64 or 128; 0 = library default). */
#define RD_TUNE_BLOCK(threads) ((threads) == 32 ? (5 << 16) : (threads) == 64 ? (6 << 16) \
                                : (threads) == 128 ? (7 << 16) : 0)
/* OR-able tuning field for RD_VARIANT_SERIAL_REGSTATE: links whose state stays in
 * registers (8 or 16; 0 = library default). */
#define RD_TUNE_REGLINKS(links) (((links) / 4) << 20)
/* OR-able tuning field for RD_VARIANT_SERIAL_HYBRID: links whose state is kept
 * (a multiple of 4, at most RD_MAX_LINKS; 0 = library default). */
#define RD_TUNE_STORED_LINKS(links) (((links) / 4) << 20)
/* OR-able tuning field for RD_VARIANT_SERIAL_DH (FP32, n <= 32, 32-thread
 * blocks): of the stored links, the first `links` (4, 8, 12 or 16) keep their
 * state in registers instead of shared memory, so that more blocks fit per SM.
 * Needs at least that many stored links (RD_TUNE_STORED_LINKS). */
#define RD_TUNE_REG_STATE_LINKS(links) (((links) / 4) << 28)
/* OR-able tuning flag for RD_VARIANT_SERIAL_DH (the same rows as
 * RD_TUNE_REG_STATE_LINKS): stage the joint values through a ring of two
 * chunks instead of three, 48 bytes less shared memory per thread. */
#define RD_TUNE_TWO_STAGE_RING 0x8000

#define RD_MAX_LINKS 128

/*
 * rd_model_create -- upload a serial chain of n revolute joints.
 *
 *   n        number of links / joints, 1 <= n <= RD_MAX_LINKS.
 *   M        host, n*12 doubles: per link the rotation of M_i (row-major
 *            3x3) then its translation (3). (Sec. II-A, Eq. id-forward.)
 *   S        host, n*6 doubles: joint twist S_i = (v, w) in frame i; |w| = 1
 *            and w.v = 0 (revolute joint) are required.
 *   inertia  host, n*10 doubles: (m, c_x, c_y, c_z, I_xx, I_yy, I_zz, I_xy,
 *            I_xz, I_yz): mass, centre of mass in frame i, and rotational
 *            inertia about the centre of mass in frame i's axes (m > 0, the
 *            3x3 inertia positive semi-definite; a point mass is allowed).
 *   out      receives the handle.
 *
 * The arrays are copied; the caller keeps ownership. The model lives on the
 * current CUDA device, and every batch call must run with that device
 * current. Allocation happens here, never in the batch calls.
 * Errors: RD_ERR_RANGE (n), RD_ERR_ARG (null pointer, non-unit axis, pitched
 * twist, non-positive mass or inertia), RD_ERR_ALLOC, RD_ERR_CUDA.
 */
int rd_model_create(int n, const double *M, const double *S, const double *inertia,
                    rd_model **out);

/* Free a model (NULL is ignored). Must not race with work using it. */
void rd_model_destroy(rd_model *model);

/* Number of links of a model, or RD_ERR_ARG for NULL. */
int rd_model_links(const rd_model *model);

/*
 * rnea_batch -- inverse dynamics for B states of one chain:
 *     tau = ID(q, qd, qdd, V_0, dV_0, F_{n+1})   (Sec. II-A; Algorithm 1)
 *
 *   model    from rd_model_create (n links).
 *   B        batch size, B >= 0 (B == 0 is a no-op).
 *   dtype    RD_F32 or RD_F64: element type of q, qd, qdd and tau, and the
 *            arithmetic precision.
 *   q, qd, qdd  device, [B, n] row-major, contiguous, dtype elements.
 *   tau      device, [B, n] row-major output; may not alias the inputs.
 *   base     host, 18 doubles {V_0[6], dV_0[6], F_{n+1}[6]} shared by the
 *            batch, or NULL for a base at rest under gravity along -z
 *            (dV_0 = (0, 0, 9.81, 0, 0, 0), F_{n+1} = 0).
 *   variant  rd_variant value or RD_VARIANT_SCAN(L).
 *   stream   cudaStream_t to launch on.
 *
 * Errors: RD_ERR_ARG (null model/pointers with B > 0, bad variant),
 * RD_ERR_DTYPE, RD_ERR_RANGE (B < 0), RD_ERR_CUDA (launch failure).
 */
int rnea_batch(const rd_model *model, int B, int dtype, const void *q, const void *qd,
               const void *qdd, void *tau, const double *base, int variant, void *stream);

/*
 * rnea_batch_host -- rnea_batch on HOST arrays (the inverse dynamics of Sec. II-A,
 * Eqs. id-forward and id-backward); returns when tau is on the host.
 * In place: with variant RD_VARIANT_AUTO, RD_F32 data, n % 4 == 0, n <= 64 and
 * all four arrays mapped pinned host memory (cudaHostAlloc under unified
 * addressing, as pinned torch tensors are) on 16-byte boundaries, one kernel
 * reads the rows from host memory and writes tau back itself, each block moving
 * contiguous slabs (RD_RNEA_KERNEL_DH_HOST; the same recursion as rnea_batch in
 * another schedule, so tau agrees with it to FP32 rounding).
 * Staged otherwise, or with variant | RD_FLAG_HOST_COPY: q, qd, qdd are copied
 * into device buffers owned by the model (grown on demand: only this path may
 * allocate device memory; rnea_batch never does), the kernel runs, and tau is
 * copied back. Large batches are split into row chunks pipelined over three
 * streams (copies in, kernels on the caller's stream, copies out), so the
 * inbound copies of a chunk overlap the kernel of the one before. Chunks are
 * never smaller than the batch size at which AUTO switches kernels, so tau is
 * identical to rnea_batch on the same rows. Pinned host memory copies at full
 * link speed (~200 GB/s per direction on GB300).
 * Same argument meaning as rnea_batch; RD_ERR_ARG also when tau aliases an input.
 */
int rnea_batch_host(rd_model *model, int B, int dtype, const void *q, const void *qd,
                    const void *qdd, void *tau, const double *base, int variant,
                    void *stream);

/* Modes of rnea_vjp (OR-able with RD_FLAG_FAST_TRIG and RD_VJP_FLAG_JOINT_FRAMES).
 * Rows with n % 4 == 0, n <= 128 and 16-byte aligned arrays run in the
 * common-normal link frames of RD_VARIANT_SERIAL_DH, with the link constants as
 * a kernel parameter; other rows in the joint frames. */
enum rd_vjp_mode {
    RD_VJP_AUTO = 0,      /* library's choice (FP64 with a large enough workspace: store) */
    RD_VJP_STORE = 1,     /* keep the forward sweep's state in the workspace */
    RD_VJP_RECOMPUTE = 2  /* keep nothing: re-derive it by inverting the forward step */
};
/* OR-able into the mode of rnea_vjp: run the joint-frame kernel even where the
 * common-normal one applies (for comparisons). */
#define RD_VJP_FLAG_JOINT_FRAMES 0x2000
/* OR-able into the mode of rnea_vjp, for FP32 in RD_VJP_RECOMPUTE on
 * common-normal rows: split each instance between two warps, one carrying the
 * motion and the wrenches, the other the adjoints (RD_VJP_FLAG_TWO_WARPS), or
 * keep one thread per instance (RD_VJP_FLAG_ONE_THREAD). Without either, the
 * library splits chains of more than 64 links in batches of at most 8192
 * states, the case where the split measured faster. Setting both is RD_ERR_ARG. */
#define RD_VJP_FLAG_TWO_WARPS 0x800
#define RD_VJP_FLAG_ONE_THREAD 0x400
/* OR-able into the mode of rnea_vjp, for FP32 in RD_VJP_RECOMPUTE (or AUTO) on
 * whole 16-byte chunks: spread each instance over RD_VJP_LANES_OF(flags) lanes
 * (4 or 8; 8 if unset), which scan the forward recursion with the adjoint
 * weight as a third channel and the reverse recursion as affine segment maps
 * (Sec. III), for batches too small to fill the GPU with one thread per
 * instance. Without it the library picks by the batch size. */
#define RD_VJP_FLAG_LANES 0x100
#define RD_VJP_FLAG_LANES4 0x200
/* OR-able into the mode of rnea_vjp, FP32, n % 4 == 0, n <= 64, recompute or
 * AUTO: one thread per instance that keeps V, dV, Fb, cos and sin of every link
 * in the block's shared memory instead of re-deriving them in the reverse
 * sweep (no workspace). Without it the library picks by the batch size. */
#define RD_VJP_FLAG_SHARED_STATE 0x4000
/* OR-able into the mode of rnea_vjp, FP32 in RD_VJP_RECOMPUTE (or AUTO), whole
 * 16-byte chunks, n <= 64: two warps per 32 instances with the per-link state
 * in shared memory. One warp carries the motion, the wrench F and dVbar, the
 * other the adjoint weight Fb and Vbar (with its own copy of the dVbar carry);
 * they exchange nothing inside a sweep and combine their gradient terms at the
 * end. Excludes the other mapping flags. */
#define RD_VJP_FLAG_TWO_WARPS_SHARED 0x8000

/*
 * rnea_vjp -- vector-Jacobian product of inverse dynamics for B states:
 *     gq = d(w^T tau)/dq,  gqd = d(w^T tau)/dqd,  gqdd = d(w^T tau)/dqdd,
 * with tau = ID(q, qd, qdd, V_0, dV_0, F_{n+1}) (Sec. II-A). The adjoint of the
 * backward scan runs base -> tip beside the forward scan, and the adjoint of
 * the forward scan runs tip -> base beside the backward scan. The paper lists
 * gradient scans as future work (Sec. VI).
 *
 *   q, qd, qdd, w     device, [B, n] row-major, dtype elements (w = d loss / d tau).
 *   gq, gqd, gqdd     device, [B, n] outputs; distinct, not aliasing the inputs.
 *   base              as in rnea_batch (NULL = rest under gravity along -z).
 *   mode              rd_vjp_mode value, optionally | RD_FLAG_FAST_TRIG.
 *   workspace         device scratch for RD_VJP_STORE (16-byte aligned), at least
 *                     rnea_vjp_workspace_size() bytes; caller-owned; may be NULL
 *                     for RD_VJP_RECOMPUTE. Its contents are overwritten.
 *   stream            cudaStream_t.
 * Errors: RD_ERR_ARG (null/aliased pointers, workspace too small or unaligned,
 * unknown mode), RD_ERR_DTYPE, RD_ERR_RANGE, RD_ERR_CUDA. Never allocates.
 */
int rnea_vjp(const rd_model *model, int B, int dtype, const void *q, const void *qd,
             const void *qdd, const void *w, void *gq, void *gqd, void *gqdd,
             const double *base, int mode, void *workspace, size_t workspace_bytes,
             void *stream);

/* Bytes of workspace rnea_vjp needs in RD_VJP_STORE mode for B states
 * (n * 20 scalars per state). */
int rnea_vjp_workspace_size(const rd_model *model, int B, int dtype, size_t *bytes);

/* Size of the fixed scratch array behind rnea_vjp_noalloc: 32 MiB per device. */
#define RD_VJP_NOALLOC_SCRATCH_BYTES (32u << 20)

/*
 * rnea_vjp_noalloc -- rnea_vjp in RD_VJP_STORE mode with library-owned
 * scratch, for callers that cannot allocate device memory when they call (a
 * real-time loop with a no-allocation rule, a plug-in whose host framework
 * owns the memory pool). The paper has no counterpart: this is an interface
 * convenience of the library.
 *
 * The caller passes inputs and outputs exactly as for rnea_vjp. The store-mode
 * scratch comes from a file-scope device array of RD_VJP_NOALLOC_SCRATCH_BYTES
 * that every device loading the library keeps until the process exits; this
 * call allocates nothing (no cudaMalloc, no cudaFree, no allocating library
 * routine).
 *   - Limit: n * 20 * B * sizeof(dtype) must not exceed the scratch size, else
 *     RD_ERR_RANGE with a message giving both sizes (e.g. n = 32 in FP32 allows
 *     B <= 13107).
 *   - Set-up: the first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture. The address is kept for the life of the
 *     process: do not call cudaDeviceReset while the library is in use.
 *   - Sharing: all calls share the one array and it keeps the last call's
 *     contents; every slot is written before it is read, so nothing is cleared.
 *     Calls that overlap on the GPU (other streams, other threads) race on it:
 *     serialise them.
 * Other errors as for rnea_vjp.
 */
int rnea_vjp_noalloc(const rd_model *model, int B, int dtype, const void *q, const void *qd,
                     const void *qdd, const void *w, void *gq, void *gqd, void *gqdd,
                     const double *base, void *stream);

/*
 * aba_batch -- forward dynamics for B states of one chain:
 *     qdd = FD(q, qd, tau, V_0, dV_0, F_{n+1})   (Sec. II-B, Eq. fd)
 * by the articulated-body algorithm: tau_bias = ID(q, qd, 0, ...) (Eq. tau-bias),
 * the articulated-body inertias (Eq. abi), and the backward / forward linear
 * recursions of Eq. recursive-fd (the scans of Sec. III-D; Algorithm 3 without
 * its CPU stage). Arithmetic in dtype, except the articulated-inertia update
 * and the divisions by Omega_i = S_i^T J_hat_i S_i: FP64 for RD_F64 data (and
 * with RD_ABA_FP64_UPDATE); double-float (about 48 bits) for RD_F32 data. For
 * RD_F32 data the bias sweeps run in double-float for n >
 * RD_ABA_EXTENDED_BIAS_LINKS (see RD_ABA_EXTENDED_BIAS).
 *
 *   q, qd, tau  device, [B, n] row-major inputs; qdd device [B, n] output.
 *   base        as in rnea_batch.
 *   status      device int[B] or NULL: RD_WARN_SINGULAR when an Omega_i <= 0 or a
 *               non-finite qdd appeared for that instance, else 0.
 *   workspace   device scratch of at least aba_workspace_size() bytes, 16-byte
 *               aligned, caller-owned; contents overwritten.
 * Errors: RD_ERR_ARG (null/aliased pointers, small or unaligned workspace),
 * RD_ERR_DTYPE, RD_ERR_RANGE, RD_ERR_CUDA. Never allocates.
 */
int aba_batch(const rd_model *model, int B, int dtype, const void *q, const void *qd,
              const void *tau, void *qdd, const double *base, int *status, int flags,
              void *workspace, size_t workspace_bytes, void *stream);

/* Bytes of workspace aba_batch needs for B states with these flags. */
int aba_workspace_size(const rd_model *model, int B, int dtype, int flags, size_t *bytes);

/*
 * jsiia_batch -- forward dynamics for B states by joint-space-inertia inversion
 * (Sec. III-C, Eqs. tau-bias and JSIinv; Algorithm 2), for n <= 32: the n
 * columns M_{.,j}(q) = ID(q, 0, delta_j, 0, 0, 0) and tau_bias = ID(q, qd, 0, ...)
 * evaluated in parallel (one lane each), then a Cholesky solve of
 * M qdd = tau - tau_bias. Columns and bias in dtype; factorisation and solve in
 * FP64. One warp per instance; no workspace.
 *   q, qd, tau  device, [B, n] inputs; qdd device [B, n] output.
 *   status      device int[B] or NULL: RD_WARN_SINGULAR when a pivot is not
 *               positive or qdd is not finite.
 * Errors: RD_ERR_RANGE (n > 32 or B < 0), RD_ERR_ARG, RD_ERR_DTYPE, RD_ERR_CUDA.
 */
int jsiia_batch(const rd_model *model, int B, int dtype, const void *q, const void *qd,
                const void *tau, void *qdd, const double *base, int *status, void *stream);

/* ---------------------------------------------------------------------------
 * Fleets: many chains of different lengths, mixed requests in one call.
 * ------------------------------------------------------------------------- */
typedef struct rd_fleet rd_fleet;
typedef struct rd_plan rd_plan;

enum rd_request_kind { RD_REQ_ID = 0, RD_REQ_FD = 1 };
enum rd_schedule {
    RD_SCHED_PERSISTENT = 0, /* one launch; resident CTAs pull sorted requests, 32 per warp,
                                from an atomic counter the call resets first */
    RD_SCHED_PER_GROUP = 1   /* one launch per run of equal (kind, n), spread over 8
                                side streams forked from and joined into the call's stream */
};
/* OR-able with the schedule: forward-dynamics requests of an RD_F32 plan run their
 * inertia updates and solves in FP64 instead of the default double-float
 * arithmetic (as RD_ABA_FP64_UPDATE for aba_batch). */
#define RD_FLEET_FP64_UPDATE 0x10
/* Tuning word for RD_SCHED_PERSISTENT: threads per CTA = 2^t, CTAs per SM = c
 * (0 = library default: 128 threads, 4 CTAs per SM). */
#define RD_FLEET_TUNE(log2_threads, ctas_per_sm) (((log2_threads) << 8) | (ctas_per_sm))
/* OR-ed into the tune word of the persistent schedule: groups of 32 sorted
 * requests that start with a forward-dynamics chain of at least min_links links
 * (1..127) run two warps per 32 requests, one on the articulated-inertia
 * recursion and one on the rest (as RD_ABA_TWO_WARPS); threads per block must
 * then be a multiple of 64 up to 448. */
#define RD_FLEET_TWO_WARPS(min_links) ((min_links) << 16)
/* As RD_FLEET_TWO_WARPS with three warps per 32 requests (as RD_ABA_THREE_WARPS);
 * the tune word's 2^t threads per block then name 2^t / 64 triples (t = 6 or 7:
 * 96 or 192 threads). */
#define RD_FLEET_THREE_WARPS(min_links) (((min_links) << 16) | (1 << 24))

/*
 * rd_fleet_create -- upload nrobots chains (Sec. II-A model per robot).
 *   n        host int[nrobots], 1 <= n[r] <= RD_MAX_LINKS.
 *   M, S, inertia  host, the robots' arrays (as for rd_model_create) concatenated
 *            in robot order: sum(n) * 12, * 6 and * 10 doubles.
 * Allocates device memory; errors as for rd_model_create (message names the robot).
 */
int rd_fleet_create(int nrobots, const int *n, const double *M, const double *S,
                    const double *inertia, rd_fleet **out);
void rd_fleet_destroy(rd_fleet *fleet);

/*
 * rd_plan_create -- a fixed set of R requests on a fleet, for data type dtype:
 * the group-level batching of many robots (Sec. I), each request inverse
 * dynamics (Sec. II-A) or forward dynamics (Sec. II-B).
 *   robot    host int[R]: robot of each request.
 *   kind     host int[R]: RD_REQ_ID (tau from q, qd, qdd) or RD_REQ_FD (qdd from
 *            q, qd, tau; articulated-body algorithm as aba_batch: inertia updates
 *            and solves in double-float arithmetic for RD_F32 plans, or FP64 with
 *            RD_FLEET_FP64_UPDATE, and FP64 for RD_F64 plans).
 * Joint data of a call is ragged: request r uses elements [off_r, off_r + n_r)
 * of every array, off_r the running sum of n over earlier requests
 * (rd_plan_offsets). The plan sorts requests (forward dynamics first, then by
 * decreasing n) and allocates its device index arrays, work counter and
 * forward-dynamics workspace here; fleet_batch allocates nothing.
 */
int rd_plan_create(const rd_fleet *fleet, int R, const int *robot, const int *kind, int dtype,
                   rd_plan **out);
void rd_plan_destroy(rd_plan *plan);
/* Length of each ragged data array (sum of n over the requests), -1 for NULL. */
long long rd_plan_total_joints(const rd_plan *plan);
/* Host copy of the R request offsets. */
int rd_plan_offsets(const rd_plan *plan, long long *off);
/* Number of (kind, n) groups, i.e. launches of RD_SCHED_PER_GROUP. */
int rd_plan_groups(const rd_plan *plan);

/*
 * fleet_batch -- evaluate every request of a plan: tau = ID(q, qd, qdd) of
 * Sec. II-A or qdd = FD(q, qd, tau) of Sec. II-B (Eqs. abi, recursive-fd).
 *   q, qd    device, ragged inputs (plan dtype).
 *   in2      device: qdd for RD_REQ_ID requests, tau for RD_REQ_FD requests.
 *   out      device: tau for RD_REQ_ID, qdd for RD_REQ_FD; must not alias inputs.
 *   base     host {V_0, dV_0, F_{n+1}} for every request (F_{n+1} in each robot's
 *            frame n), or NULL for rest under gravity along -z.
 *   status   device int[R] or NULL: RD_WARN_SINGULAR for a forward-dynamics
 *            request that met Omega_i <= 0 or a non-finite qdd.
 *   schedule rd_schedule, optionally | RD_FLEET_FP64_UPDATE; tune: RD_FLEET_TUNE(...) or 0.
 * Concurrent calls on one plan race on its counter and workspace.
 */
int fleet_batch(const rd_plan *plan, const void *q, const void *qd, const void *in2, void *out,
                const double *base, int *status, int schedule, int tune, void *stream);

/*
 * rd_measure_fma_peak -- diagnostic, outside the paper's method: measured
 * fused-multiply-add throughput of the current device in TFLOP/s (FMA = 2
 * flops) for RD_F32 or RD_F64, from independent FMA chains on every SM.
 * Allocates a small device buffer and synchronizes the stream.
 */
int rd_measure_fma_peak(int dtype, double *tflops, void *stream);

/*
 * rd_joint_trig -- diagnostic, outside the paper's method: the FP32 sine and
 * cosine that the common-normal-frame kernels evaluate for each joint angle
 * (Cody-Waite reduction by pi/2 and fitted polynomials on the FMA pipe; with
 * flags & RD_FLAG_FAST_TRIG, the special-function-unit approximation).
 *   x, s, c  device float[count]: angles in radians in, sin and cos out.
 *   stream   cudaStream_t. Asynchronous; never allocates.
 * Errors: RD_ERR_RANGE (count < 0), RD_ERR_ARG (null pointer), RD_ERR_CUDA.
 */
int rd_joint_trig(int flags, const float *x, float *s, float *c, int count, void *stream);

/*
 * rd_joint_trig_df -- diagnostic, outside the paper's method: the sine and
 * cosine that RD_VARIANT_SERIAL_DF evaluates for each FP64 joint angle, in
 * double-float arithmetic (Cody-Waite reduction by pi/2 in FP64, Taylor series
 * with inverse-factorial coefficients), returned as doubles (hi + lo).
 *   x, s, c  device double[count]: angles in radians in, sin and cos out.
 *   stream   cudaStream_t. Asynchronous; never allocates.
 * Errors: RD_ERR_RANGE (count < 0), RD_ERR_ARG (null pointer), RD_ERR_CUDA.
 */
int rd_joint_trig_df(const double *x, double *s, double *c, int count, void *stream);

/*
 * rd_rnea_last_config -- the kernel the calling thread's last rnea_batch call
 * launched (a diagnostic for tuning and benchmarks):
 *   kernel        an rd_variant value naming the kernel family (RD_VARIANT_SERIAL,
 *                 ..._RECOMPUTE, ..._RECOMPUTE_CS, ..._REGSTATE, ..._HYBRID,
 *                 RD_VARIANT_SERIAL_DH, ..._DH_RECOMPUTE with shared-memory
 *                 constants, RD_VARIANT_SCAN(L)) or RD_RNEA_KERNEL_DH_PARAM for
 *                 the common-normal kernel with its constants as a kernel
 *                 parameter, RD_RNEA_KERNEL_DH_TMEM for its variant with state in
 *                 tensor memory;
 *   block         threads per block;
 *   stored_links  links whose full backward-sweep state the kernel keeps.
 * All 0 before the first launch on this thread. Errors: RD_ERR_ARG (null output).
 */
#define RD_RNEA_KERNEL_DH_PARAM 0x206
#define RD_RNEA_KERNEL_DH_TMEM 0x208
#define RD_RNEA_KERNEL_DH_HOST 0x209 /* rnea_batch_host reading mapped host arrays */
int rd_rnea_last_config(int *kernel, int *block, int *stored_links);
/* Where the last launch of the common-normal kernel with stored state kept it:
 * how many of the stored links in registers (RD_TUNE_REG_STATE_LINKS, or the
 * library's choice), and how many chunks of joint values its staging ring
 * held (3, or 2 with RD_TUNE_TWO_STAGE_RING or the library's choice); both 0
 * after any other kernel. Errors: RD_ERR_ARG (null output). */
int rd_rnea_last_state_layout(int *register_links, int *ring_chunks);

/* Message for the last error on the calling thread ("" if none). */
const char *rd_last_error(void);

/* Library ABI version (major * 100 + minor). */
int rd_version(void);

#ifdef __cplusplus
}
#endif

#endif /* RDYN_H */
