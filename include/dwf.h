/*
 * dwf.h -- C-ABI of the GB300 (sm_103a) even-odd preconditioned domain-wall fermion solver.
 *
 * The library applies and inverts the 5D domain-wall operator of Chiu, Hsieh, Mao, Ogawa,
 * "GPU-Based Conjugate Gradient Solver for Lattice QCD with Domain-Wall Fermions"
 * (Lattice 2010):
 *
 *   D(mq) = D_w (omega + sigma L) + (1 - L)                                   (Eq. 1, Eq. 5)
 *   D_w   = Wilson operator with the -m0 term, d = 4                          (Eq. 2)
 *   L     = P+ L+ + P- L-,  (L+)_{s,s-1} = 1, (L+)_{1,Ns} = -mq/(2 m0)        (Eq. 3-4)
 *   M5    = [ (d - m0) + omega^{-1/2} (1 - L)(1 + cL)^{-1} omega^{-1/2} ]^{-1} (Eq. 8)
 *   C     = 1 - M5 D_w^{p,1-p} M5 D_w^{1-p,p}  on Schur parity p              (Eq. 11)
 *
 * and solves C C^dagger x = b (Sec. 2.2) with a conjugate gradient (Algorithm 1) whose
 * inner iterations run in FP32 (or 16-bit storage) and whose restarts recompute the true
 * residual in FP64: reliable updates that keep the search direction, switching to defect
 * correction (Algorithm 2) when reliable updates stop converging (Sec. 2.3).
 *
 * Conventions (readings of what the paper leaves open):
 *   dims = {Nx, Ny, Nz, Nt}, every extent even and >= 2; periodic boundaries.
 *   Host spinor layout (Sec. 3.1): real index c + 24 s + 24 Ns site with
 *   site = x + Nx (y + Ny (z + Nz t)), c = reim + 2 (colour + 3 spin), s = 0..Ns-1.
 *   A full 5D field holds 24 * Ns * Nx*Ny*Nz*Nt doubles.
 *   Host gauge layout: U_mu(x)_{ab} at complex index ((site*4 + mu)*3 + a)*3 + b,
 *   mu = 0..3 for x, y, z, t (72 doubles per site).
 *   Gamma matrices: chiral basis, gamma_k = [[0, -i sigma_k], [i sigma_k, 0]],
 *   gamma_4 = [[0, 1], [1, 0]], gamma_5 = gamma_1 gamma_2 gamma_3 gamma_4 = diag(1,1,-1,-1);
 *   P+ acts on spins 0,1 and P- on spins 2,3.
 *   Parity of a site: (x + y + z + t) mod 2, 0 = even, 1 = odd.  D_w^{EO} maps odd to
 *   even sites, D_w^{OE} even to odd (block positions of Eq. 6).
 *
 * Ownership: the caller owns every host buffer and every device buffer it passes; the
 * library copies in and out and never frees caller memory.  A dwf_ctx owns its device
 * state (gauge copies, matrices, work vectors) and releases it in dwf_destroy.  A
 * context is used by one host thread at a time; its calls are ordered on one CUDA stream.
 *
 * Errors: every call returns a dwf_status; nothing aborts and no exception crosses the
 * boundary.  dwf_last_error(ctx) describes the last failure on that context.
 */
#ifndef DWF_H
#define DWF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dwf_ctx dwf_ctx;

typedef enum {
    DWF_OK = 0,
    DWF_EINVAL = 1,   /* invalid argument (odd extent, Ns < 1, omega_s <= 0, m0 outside (0,2), ...) */
    DWF_ENOMEM = 2,   /* device or host allocation failed, or a budget would be exceeded */
    DWF_ENOCONV = 3,  /* solver reached max_iter without meeting tol (stats still filled) */
    DWF_EBUSY = 4,    /* no free slot (server) */
    DWF_EAGAIN = 5,   /* poll: request not finished yet */
    DWF_ETIMEOUT = 6, /* a bounded device-side wait gave up (kernel error word set) */
    DWF_ECUDA = 7,    /* a CUDA runtime call failed; see dwf_last_error */
    DWF_ENOGAUGE = 8, /* operator used before dwf_load_gauge */
    DWF_ECOMM = 9     /* a dwf_part_comm callback reported failure */
} dwf_status;

/* operators of dwf_apply_eo */
enum {
    DWF_OP_DEO = 0,   /* out_even = D_w^{EO} in_odd   (Eq. 12, hopping term only) */
    DWF_OP_DOE = 1,   /* out_odd  = D_w^{OE} in_even  (Eq. 12) */
    DWF_OP_M5 = 2,    /* out_p = M5 in_p   (Eq. 8), on the sites of `parity` */
    DWF_OP_M5T = 3,   /* out_p = M5^T in_p */
    DWF_OP_C = 4,     /* out_p = C in_p    (Eq. 11) on Schur parity p = `parity` */
    DWF_OP_CDAG = 5,  /* out_p = C^dagger in_p */
    DWF_OP_CCDAG = 6, /* out_p = C C^dagger in_p */
    DWF_OP_DFULL = 7, /* out = D(mq) in on the whole lattice (Eq. 1 / Eq. 5) */
    DWF_OP_DW = 8     /* out = D_w in on every s-slice, whole lattice (Eq. 2) */
};

/* arithmetic of an operator application or of the inner CG */
enum {
    DWF_PREC_F64 = 0,  /* FP64 storage and arithmetic */
    DWF_PREC_F32 = 1,  /* FP32 storage and arithmetic */
    DWF_PREC_F16 = 2,  /* fp16 spinors with a per-(site,s) FP32 norm, 12-real fp16 links, FP32 arithmetic */
    DWF_PREC_BF16 = 3  /* bf16 spinors with a per-(site,s) FP32 norm, 12-real bf16 links, FP32 arithmetic */
};

/* restart policy of the mixed-precision CG (Sec. 2.3) */
enum {
    DWF_MODE_AUTO = 0,     /* reliable updates; switch to defect correction if they stop converging,
                              and from 16-bit to FP32 inner iterations if defect correction stops too */
    DWF_MODE_RELIABLE = 1, /* keep p across restarts (reliable updates) */
    DWF_MODE_DEFECT = 2    /* reset p := r at every restart (defect correction, Algorithm 2) */
};

/* which system dwf_solve solves */
enum {
    DWF_SYS_FULL = 0,   /* D psi = eta on the whole lattice, via Eq. 10 (source prep + CG + reconstruction) */
    DWF_SYS_NORMAL = 1  /* C C^dagger x = b on the sites of schur_parity (the HMC use, Sec. 2.2) */
};

typedef struct {
    double tol;        /* stop when |b - C C^dag x| <= tol |b| in FP64 (default 1e-10) */
    double delta;      /* reliable-update trigger: restart when |r| < delta * max|r| since the
                          last restart; <= 0 selects the default of the inner precision:
                          0.3 for fp16, 0.01 otherwise */
    int max_iter;      /* cap on inner CG iterations (default 100000) */
    int inner_prec;    /* DWF_PREC_* of the inner CG (default DWF_PREC_F32) */
    int mode;          /* DWF_MODE_* (default DWF_MODE_AUTO) */
    int system;        /* DWF_SYS_* (default DWF_SYS_FULL) */
    int schur_parity;  /* parity of the Schur complement, 0 or 1 (default 1, the paper's odd sites) */
    int check_every;   /* inner iterations between host polls of the device flags (default 8) */
    int use_graph;     /* capture each batch of inner iterations in a CUDA graph (default 1) */
    int profile;       /* record CUDA events around every kernel class (default 0) */
    int stall_iters;   /* restart, resetting the search direction, when |r| has not reached a
                          new minimum for this many inner iterations; <= 0 selects 500 */
    int schur_target_pct; /* full system: the Schur residual aims at this percentage of tol
                          (<= 0 selects 50); a system whose full residual |eta - D psi| / |eta|
                          still misses tol continues once with a tightened target */
    int use_x0;        /* warm start: sol holds an initial guess x0 on entry (Algorithm 2
                          starting from x_hat = x0); the FP64 residual rhs - A x0 is solved
                          for the correction, so the result meets tol relative to |rhs|.
                          Normal system: x0's sites of the other parity are ignored.
                          A source or guess with a non-finite entry gives DWF_EINVAL.
                          Right-hand sides of a batch are then solved one after another */
    int no_autotune;   /* 0 (default): the first solve of a (device, inner precision, Ns,
                          volume class) times the candidate launch shapes of the inner hop
                          kernels on its own fields and keeps the fastest for the process
                          (results agree with other shapes to rounding: only the order of
                          the reductions' block sums differs); 1: the default shapes */
    int reserved[2];
} dwf_solve_params;

/* kernel classes timed when params.profile != 0 */
enum {
    DWF_KC_HOP_M5 = 0,     /* inner hop + M5 epilogue (t = M5^T D w, u = M5 D q) */
    DWF_KC_HOP_XPAY = 1,   /* inner hop + (p - g5 D t) epilogue + norm */
    DWF_KC_HOP_UPDATE = 2, /* inner hop + M5 + CG update (r, x) + norm */
    DWF_KC_SMIX_P = 3,     /* inner p = r + beta p and w = M5^T g5 p */
    DWF_KC_F64 = 4,        /* FP64 restart operator, source preparation, reconstruction */
    DWF_KC_OTHER = 5,      /* packing, conversions, norms */
    DWF_KC_COUNT = 6
};

typedef struct {
    int iters;             /* inner CG iterations */
    int restarts;          /* FP64 true-residual recomputations */
    int mode_used;         /* DWF_MODE_RELIABLE or DWF_MODE_DEFECT at the end */
    int converged;         /* 1 when true_res <= tol */
    double true_res;       /* |b - C C^dag x| / |b| in FP64 */
    double true_res_full;  /* |eta - D psi| / |eta| in FP64 (DWF_SYS_FULL only, else 0) */
    double flops;          /* counted flops: per 5D half-site, CG iteration 5472 + 192 Ns, FP64 restart
                              5328 + 192 Ns, source preparation and reconstruction 5160 + 384 Ns */
    double time_ms;        /* device time of the whole call, CUDA events on its stream */
    double class_ms[DWF_KC_COUNT];   /* per kernel class, when profiling */
    int class_launches[DWF_KC_COUNT];
    long long kernel_launches;       /* kernels this call launched (graph nodes included) */
    double bytes_hop_m5;             /* algorithmic bytes of one DWF_KC_HOP_M5 launch */
    int inner_prec_used;             /* DWF_PREC_* of the inner CG at the end */
    int escalations;                 /* AUTO mode: 16-bit inner CG replaced by FP32 (0 or 1) */
    double reserved[2];
} dwf_solve_stats;

/* Fill p with the defaults listed above. */
void dwf_solve_params_default(dwf_solve_params *p);

/* Create a context for one lattice and one set of 5th-dimension parameters (Eq. 1-4).
 * dims: host array {Nx,Ny,Nz,Nt}; Ns >= 1 and <= 64; 0 < m0 < 2; mq >= 0;
 * omega, sigma: host arrays of Ns doubles, omega_s > 0 (copied).  Uses the current
 * CUDA device.  On success *out receives the context. */
dwf_status dwf_create(const int dims[4], int Ns, double m0, double mq, const double *omega,
                      const double *sigma, dwf_ctx **out);

/* Release every device and host resource of ctx (NULL is accepted). */
dwf_status dwf_destroy(dwf_ctx *ctx);

/* Load the gauge field from a host array in the host gauge layout (72 * V4 doubles).
 * The links must be SU(3) for the 12-real 16-bit form to be exact. */
dwf_status dwf_load_gauge(dwf_ctx *ctx, const double *U);
/* Same from a device array (caller-owned, host gauge layout), ordered on `stream`
 * (a cudaStream_t; NULL = the context's stream). */
dwf_status dwf_load_gauge_dev(dwf_ctx *ctx, const double *d_U, void *stream);

/* Gauge fields shared by handle.  dwf_gauge_create copies a gauge field (host gauge layout,
 * 72 * V4 doubles; dwf_gauge_create_dev: a caller-owned device array, read after the work
 * already queued on `stream`) to the CUDA device current at the call; the object keeps that
 * FP64 copy and builds the doubled per-parity link forms of each precision once, on the
 * first use by any context.  dwf_attach_gauge makes a context of the same lattice use it
 * instead of a private copy (its previous gauge, private or shared, is released); any
 * number of contexts -- different Ns, masses and weights -- can share one gauge object.
 * dwf_gauge_release drops the caller's reference; the object is freed when no context uses
 * it any more.  A later dwf_load_gauge on a context detaches it again.  Links must be SU(3)
 * for the 12-real 16-bit forms.  Errors: DWF_EINVAL (odd extent, lattice or device of the
 * context and the gauge differ), DWF_ENOMEM, DWF_ECUDA. */
typedef struct dwf_gauge dwf_gauge;
dwf_status dwf_gauge_create(const int dims[4], const double *U, dwf_gauge **out);
dwf_status dwf_gauge_create_dev(const int dims[4], const double *d_U, void *stream, dwf_gauge **out);
dwf_status dwf_gauge_release(dwf_gauge *gauge);
dwf_status dwf_attach_gauge(dwf_ctx *ctx, dwf_gauge *gauge);

/* Apply operator `op` (DWF_OP_*) in precision `prec` (DWF_PREC_*) to a full-lattice host
 * array `in` (24*Ns*V4 doubles, host layout) and write the full-lattice host array
 * `out`.  Only the sites the operator reads are used from `in`; every site the
 * operator does not write is set to 0 in `out`.  `parity` is the Schur parity for
 * M5/M5T/C/CDAG/CCDAG and is ignored otherwise.  in and out must not overlap. */
dwf_status dwf_apply_eo(dwf_ctx *ctx, int op, int prec, int parity, const double *in, double *out);
/* Same with caller-owned device arrays in the host layout, ordered on `stream`. */
dwf_status dwf_apply_eo_dev(dwf_ctx *ctx, int op, int prec, int parity, const double *d_in,
                            double *d_out, void *stream);

/* Solve nrhs systems with the same operator together (e.g. the 12 spin-colour point
 * sources of a propagator, Sec. 2.2's valence use).  rhs and sol hold nrhs arrays of the
 * dwf_solve layout one after another; stats, if not NULL, receives nrhs entries.  Every
 * right-hand side has its own CG scalars, restarts and convergence (Algorithm 1-2, Sec. 2.3);
 * all of them advance in the same kernel launches (one grid row per right-hand side) and the
 * same CUDA graph.  As for a single full-system solve, a right-hand side whose full residual
 * misses tol continues once with a tighter Schur target; the 16-bit-to-FP32 escalation of
 * AUTO mode applies to single solves only.  Returns the
 * first failure among the right-hand sides (DWF_ENOCONV if any did not converge). */
dwf_status dwf_solve_batch(dwf_ctx *ctx, int nrhs, const double *rhs, double *sol,
                           const dwf_solve_params *params, dwf_solve_stats *stats);
/* Same with caller-owned device arrays, ordered on `stream`. */
dwf_status dwf_solve_batch_dev(dwf_ctx *ctx, int nrhs, const double *d_rhs, double *d_sol,
                               const dwf_solve_params *params, dwf_solve_stats *stats, void *stream);

/* Solve a ragged set: one system on each of n distinct contexts of one device, which may
 * differ in lattice, Ns, masses and weights (e.g. one gauge field shared by handle, eight
 * (Ns, mq) pairs), with the same params (use_x0 not allowed).  rhs[k] and sol[k] are
 * arrays of the dwf_solve layout of context k; stats, if not NULL, receives n entries, each
 * time_ms spanning that system's own begin and end.  Every system follows Algorithm 1-2 with
 * its own scalars, restarts and convergence (Sec. 2.3), and the same kernels as it would
 * alone, so each solution equals its single solve bit for bit; each interval of check_every
 * inner iterations of all unfinished systems is one CUDA graph with a branch per context, so
 * the systems' kernels run concurrently, and the restarts between intervals run on each
 * context's own stream.  Errors about the set as a whole (duplicate contexts, contexts on
 * different devices) are reported on ctxs[0]; those of one system on its context.  Returns
 * the first failure (DWF_ENOCONV if any system did not converge).  n: 1..256. */
dwf_status dwf_solve_ragged(int n, dwf_ctx *const *ctxs, const double *const *rhs, double *const *sol,
                            const dwf_solve_params *params, dwf_solve_stats *stats);
/* Same with caller-owned device arrays; the set starts after, and `stream` continues after
 * it (NULL: ctxs[0]'s stream). */
dwf_status dwf_solve_ragged_dev(int n, dwf_ctx *const *ctxs, const double *const *d_rhs, double *const *d_sol,
                                const dwf_solve_params *params, dwf_solve_stats *stats, void *stream);

/* Quark propagator from the point x0 (the valence use of Sec. 2.2): the 12 spin-colour
 * point sources are solved in one batch (dwf_solve_batch, DWF_SYS_FULL) and the 4D quark
 * field is read off the two walls.  Conventions (the paper fixes none): source (beta, b)
 * carries a 1 in spin beta, colour b at x0 on the s-slice of its chirality's wall -- s = 0
 * for P+ (spins 0,1), s = Ns-1 for P- (spins 2,3) -- and q(x) = P- psi(x, 0) + P+ psi(x, Ns-1)
 * (L moves P+ components up and P- components down in s, Eq. 3-4).
 * prop receives V4 * 144 complex numbers, prop[site][alpha][a][beta][b] = q_{alpha a}(site)
 * of source (beta, b), re/im interleaved.  stats, if not NULL, receives 12 entries. */
dwf_status dwf_propagator(dwf_ctx *ctx, const int x0[4], const dwf_solve_params *params, double *prop,
                          dwf_solve_stats *stats);
/* Same with a caller-owned device output, ordered on `stream`. */
dwf_status dwf_propagator_dev(dwf_ctx *ctx, const int x0[4], const dwf_solve_params *params, double *d_prop,
                              dwf_solve_stats *stats, void *stream);

/* Allocation-free variant of dwf_apply_eo_dev (the paper has no counterpart: it is a
 * service for callers that cannot let a library allocate device memory -- applications
 * whose device memory is owned by their own pool allocator, such as a framework's caching
 * allocator that already holds the GPU's memory, or held to a fixed budget decided at
 * start-up -- and for paths that must not meet the device-wide synchronisation that a
 * cudaMalloc or cudaFree can bring).
 * Applies DWF_OP_DEO, DOE, M5, M5T, C, CDAG or CCDAG exactly as dwf_apply_eo_dev does, with
 * the same arguments, but takes every work field, the scalar block and the reduction
 * scratch from one static device array of 64 MiB compiled into the library (held on every
 * GPU that loads the library until the process exits) and calls no cudaMalloc, cudaFree or
 * other allocating routine.  The caller still passes the input and output arrays.  Limits
 * and behaviour:
 *   - five work fields plus the partial sums must fit in 64 MiB: about 5 * 24 * Ns * V4/2
 *     reals of the precision (FP32: Ns * V4/2 <= ~135,000; FP64: <= ~67,000, e.g. 8^4 x 16);
 *     larger lattices return DWF_EINVAL with the byte count in dwf_last_error;
 *   - the gauge field of `prec` must already exist (dwf_load_gauge builds FP64 and FP32; one
 *     dwf_apply_eo_dev call builds a 16-bit form), else DWF_EINVAL;
 *   - set-up: the first call on a context looks up the array's device address
 *     (cudaGetSymbolAddress) with the context's device current;
 *   - the call returns when its work is done: it synchronises `stream` and copies the
 *     kernels' 4-byte error word to the host (DWF_ETIMEOUT if a bounded device-side wait
 *     gave up);
 *   - every call shares the one array, which keeps the last call's contents; the call clears
 *     what must start at zero itself.  Calls that overlap on the GPU (two streams, two
 *     contexts, or two host threads) race on the array and must be serialised by the
 *     caller.  The context's own scratch is not used, so other calls on the context do not
 *     touch the array. */
dwf_status dwf_apply_eo_dev_static(dwf_ctx *ctx, int op, int prec, int parity, const double *d_in,
                                   double *d_out, void *stream);

/* 4D domain decomposition (not part of the paper's solver, which runs on one GPU; Sec. 1
 * mentions the GPU cluster its collaboration runs on).  The lattice global_dims is cut into
 * grid[0] x grid[1] x grid[2] x grid[3] blocks; each block's extents global_dims/grid must be
 * even and >= 2.  A part context (dwf_create_part; coord = its block in the grid) holds the
 * block's sites plus one halo slot per opposite-parity site beyond each cut face.  Before
 * every hop each part packs the spin projection of its cut faces (Eq. 12 with the
 * projection of Sec. 3.2: 12 reals per (site, s), half a spinor) and the packed faces are
 * copied to the neighbouring parts' halos.  dwf_load_gauge_part takes the global gauge field
 * (host gauge layout of the whole lattice, 72 * V4_global doubles) and keeps the block's
 * links.  dwf_part_apply applies DWF_OP_DEO, DOE, C, CDAG or CCDAG (precision prec, Schur
 * parity `parity`) to a global full-lattice host array `in`, the parts -- every block of the
 * grid exactly once, in any order, on one device or several -- exchanging faces between
 * the hops, and writes the global result to `out` (sites of the other parity set to 0).
 * Other calls (dwf_apply_eo*, dwf_solve*, dwf_propagator*) refuse a part context with
 * DWF_EINVAL.  Errors: DWF_EINVAL (invalid decomposition, parts of different lattices or
 * operators, a missing or repeated block), DWF_ENOGAUGE, DWF_ENOMEM, DWF_ECUDA. */
typedef struct {
    int global_dims[4];   /* whole lattice, Nx, Ny, Nz, Nt */
    int grid[4];          /* blocks per direction */
    int coord[4];         /* this part's block, 0 <= coord[mu] < grid[mu] */
} dwf_partition;
dwf_status dwf_create_part(const dwf_partition *part, int Ns, double m0, double mq, const double *omega,
                           const double *sigma, dwf_ctx **out);
dwf_status dwf_load_gauge_part(dwf_ctx *ctx, const double *U);
dwf_status dwf_part_apply(int nparts, dwf_ctx *const *parts, int op, int prec, int parity, const double *in,
                          double *out);
/* Solve across the parts: the same system as dwf_solve (params->system: D psi = eta with
 * rhs = eta, or C C^dag x = b on params->schur_parity) for a global full-lattice host rhs,
 * the solution written to the global host array sol.  Inner CG (Algorithm 1) in
 * params->inner_prec with FP64 reliable updates (Sec. 2.3: restart when |r| falls by
 * params->delta, default 0.3 for fp16 and 0.01 otherwise, or reaches the target), every reduction summed over the
 * parts in FP64 (the allreduce of a multi-GPU run: 2 per iteration), faces exchanged before
 * every hop.  The host steers each iteration (no CUDA graphs) and a full solve takes no
 * tightened second pass: DWF_ENOCONV if |eta - D psi| / |eta| misses tol.  stats (if not
 * NULL): iterations, restarts, true residuals (FP64), counted flops, host wall time. */
dwf_status dwf_part_solve(int nparts, dwf_ctx *const *parts, const double *rhs, double *sol,
                          const dwf_solve_params *params, dwf_solve_stats *stats);

/* The transport between parts held by different processes (one part each, e.g. one per
 * GPU): the library packs its part's cut faces and takes its block's sums, the caller moves
 * them.  Every part calls each callback the same number of times in the same order (they
 * are collective), from the thread of the library call.
 *   exchange: for each k = 2 mu + side with bytes[k] > 0 (direction mu cut; side 0: the face
 *     x_mu = 0, 1: the face x_mu = L_mu - 1 of the local block), send the bytes[k] bytes at
 *     send[k] to the part on that side (grid coordinate coord[mu] - 1 or + 1, periodic), and
 *     receive into recv[k] the bytes[k] bytes that this part's neighbour on that side sends
 *     towards it (its face k ^ 1).  send and recv are pinned host memory owned by the library
 *     and valid for the call; a grid of 2 along mu makes both neighbours the same part.
 *   allreduce: replace v[0..n) by its sum over all parts, identical on every part.
 * Each returns 0 on success; any other value fails the library call with DWF_ECOMM.  A part
 * whose call fails before a collective step (an invalid argument, a missing gauge field)
 * leaves the others waiting in that step: the transport's own timeout has to end their wait
 * (and return non-zero). */
typedef struct {
    void *user;
    int (*exchange)(void *user, const void *const *send, void *const *recv, const size_t *bytes);
    int (*allreduce)(void *user, double *v, int n);
} dwf_part_comm;
/* dwf_part_apply for this part alone, the others reached through comm: in and out are this
 * part's block in the host layout of its local extents (global_dims / grid, x fastest). */
dwf_status dwf_part_apply_comm(dwf_ctx *part, const dwf_part_comm *comm, int op, int prec, int parity,
                               const double *in, double *out);
/* dwf_part_solve for this part alone, the others reached through comm: rhs and sol are this
 * part's block in the host layout of its local extents.  Every decision (restart, convergence)
 * is taken on allreduced sums, so iterations, residuals and the status are the same on every
 * part; with two parts the result equals dwf_part_solve's bit for bit. */
dwf_status dwf_part_solve_comm(dwf_ctx *part, const dwf_part_comm *comm, const double *rhs, double *sol,
                               const dwf_solve_params *params, dwf_solve_stats *stats);

/* The launch shape the autotuner chose for inner-CG kernel class `kclass` (DWF_KC_HOP_M5,
 * DWF_KC_HOP_XPAY or DWF_KC_HOP_UPDATE) at precision `prec` (FP32, F16, BF16) for this
 * context's Ns and volume on its device: *threads per CTA and *persistent (1: a grid of the
 * CTAs resident at once walking all tiles; 0: one tile per CTA).  DWF_OK when tuned,
 * DWF_EAGAIN (default shape filled in) when no solve has tuned it yet, DWF_EINVAL for other
 * classes or precisions. */
dwf_status dwf_tuned_shape(dwf_ctx *ctx, int prec, int kclass, int *threads, int *persistent);

/* Solve.  DWF_SYS_FULL: rhs = eta, sol = psi (full-lattice host arrays) with D psi = eta.
 * DWF_SYS_NORMAL: rhs = b, sol = x on the sites of params->schur_parity with
 * C C^dag x = b (other sites of sol are set to 0).  params may be NULL (defaults);
 * stats may be NULL.  With params->use_x0, sol holds the initial guess on entry (it is
 * read, then overwritten with the solution).  Returns DWF_ENOCONV (with stats filled and
 * the best x written) when max_iter is reached first. */
dwf_status dwf_solve(dwf_ctx *ctx, const double *rhs, double *sol, const dwf_solve_params *params,
                     dwf_solve_stats *stats);
/* Same with caller-owned device arrays, ordered on `stream`. */
dwf_status dwf_solve_dev(dwf_ctx *ctx, const double *d_rhs, double *d_sol,
                         const dwf_solve_params *params, dwf_solve_stats *stats, void *stream);

/* ---------------------------------------------------------------------------------------
 * Serving: a request loop over many solves (not in the paper, which runs one solve at a
 * time; it is the production form of the same Schur-complement CG).  The server keeps
 * gauge ensembles resident on the device (one shared dwf_gauge per ensemble), queues
 * requests first come first served, admits a request when a slot is free and its
 * device-memory estimate fits the budget, and runs admitted solves concurrently, each on
 * its own CUDA stream, so work of requests that arrive while others run overlaps on the
 * GPU.  Queued requests of the same operator and solver settings as the admitted one join
 * it as rows of one batched solve (up to max_batch; 16-bit AUTO-mode requests run alone).
 * Contexts are cached per operator and released, least recently used first, only when a
 * new one needs the memory; releasing one does not synchronise the device.  Every solve,
 * and every row of a batch, is deterministic (fixed reduction order), so its result does
 * not depend on what else runs beside it.  Uses the CUDA device current when
 * dwf_server_create is called.
 * --------------------------------------------------------------------------------------- */
typedef struct dwf_server dwf_server;

typedef struct {
    double hbm_budget_gb;   /* device memory the server may hold for contexts and solver
                               state, GiB (default 150) */
    int max_inflight;       /* solves running at once (default 4) */
    int max_batch;          /* most requests of one operator run as one batch (0: 8) */
    int reserved[6];
} dwf_server_params;

typedef struct {
    int dims[4];            /* lattice of the request; must match its gauge ensemble */
    int Ns;
    double m0, mq;
    const double *omega;    /* Ns weights, copied at submission */
    const double *sigma;    /* Ns weights, copied at submission */
    int gauge;              /* handle from dwf_server_add_gauge */
    const double *rhs;      /* host right-hand side (full-lattice host layout), copied */
    dwf_solve_params params;/* solver settings (tol, system, inner_prec, ...); use_x0 is
                               ignored (a request carries no initial guess) */
} dwf_request;

typedef struct {
    dwf_status status;      /* status of the solve */
    dwf_solve_stats stats;
    double queue_ms;        /* submission to start of the solve */
    double latency_ms;      /* submission to completion */
} dwf_result;

typedef struct {
    long long submitted, completed, in_flight, queued;
    double p50_ms, p99_ms, mean_ms;  /* latency (submission to completion) of completed requests */
    double solves_per_s;             /* completed / (last completion - first submission) */
    double hbm_reserved_gb;          /* device-memory estimate of the admitted contexts */
    long long cancelled;             /* requests withdrawn by dwf_cancel before admission */
    long long batched;               /* requests that ran as rows of a shared batch */
} dwf_server_stats;

/* Fill p with the server defaults listed above (NULL is ignored). */
void dwf_server_params_default(dwf_server_params *p);
/* Create a server (no device work until a request runs).  params may be NULL. */
dwf_status dwf_server_create(const dwf_server_params *params, dwf_server **out);
/* Finish the running solves, drop the queued ones and free everything (NULL accepted). */
dwf_status dwf_server_destroy(dwf_server *srv);
/* Copy a gauge field (host layout, 72 * V4 doubles) to the device as a resident ensemble;
 * *handle receives its id. */
dwf_status dwf_server_add_gauge(dwf_server *srv, const int dims[4], const double *U, int *handle);
/* Queue one solve; *ticket identifies it.  The request's arrays are copied before the call
 * returns.  DWF_EINVAL for malformed requests, DWF_ENOMEM if its memory estimate alone
 * exceeds the budget. */
dwf_status dwf_submit(dwf_server *srv, const dwf_request *req, uint64_t *ticket);
/* DWF_EAGAIN while the solve is queued or running.  Once done: fills *result (if not NULL),
 * copies the solution into psi_out (if not NULL; full-lattice host layout), releases the
 * ticket and returns DWF_OK (the solve's own status is result->status).  DWF_EINVAL for an
 * unknown ticket. */
dwf_status dwf_poll(dwf_server *srv, uint64_t ticket, double *psi_out, dwf_result *result);
/* Withdraw a request that is still queued: DWF_OK (its ticket is released; a later poll
 * returns DWF_EINVAL), DWF_EBUSY if a worker has already taken it (poll it as usual),
 * DWF_EINVAL for an unknown ticket. */
dwf_status dwf_cancel(dwf_server *srv, uint64_t ticket);
/* Open (nonzero) or close admission: while closed, submitted requests queue but no worker
 * admits one (running solves continue), e.g. to drain the device or to stage a burst of
 * requests.  Servers start open. */
dwf_status dwf_server_set_admission(dwf_server *srv, int open);
/* Latency percentiles, throughput and occupancy of the server so far. */
dwf_status dwf_server_get_stats(dwf_server *srv, dwf_server_stats *stats);

/* Weights of the optimal domain-wall operator (sigma = omega in Eq. 1; Sec. 2.1 wants the
 * best chiral symmetry Ns slices allow and takes them from a cited formula it does not print).
 * Reading: the omega_s that make S(lam) = (1 - T)/(1 + T), T = prod_s (1 - omega_s lam) /
 * (1 + omega_s lam), the best uniform approximation of sgn(lam) on [lambda_min, lambda_max],
 * the range of |H_w| = |g5 D_w| the caller supplies; computed by the Remez exchange (the
 * error 1 - S alternates Ns + 1 times).  Host computation only: needs no context or GPU.
 * omega receives Ns weights, caller-owned, in decreasing order (the four-dimensional
 * operator does not depend on their order along s); delta, if not NULL, receives
 * max |1 - S| on the interval.  DWF_EINVAL: Ns outside 1..64, lambda_min <= 0,
 * lambda_max <= lambda_min, or omega NULL.  DWF_ENOCONV: the exchange did not settle (seen
 * only where delta would fall tens of orders below double precision, e.g. Ns = 64 on a
 * spectrum narrower than a factor of 2). */
dwf_status dwf_optimal_weights(int Ns, double lambda_min, double lambda_max, double *omega, double *delta);

/* Failure-detection hook, for tests.  Every wait of the hop kernels for a tile's TMA copies
 * (an mbarrier phase) is bounded; when the bound runs out the kernel sets the context's
 * error word, waits (again bounded) for the copy in flight and returns, and the call that
 * launched it returns DWF_ETIMEOUT, clears the error word and leaves the context usable.
 * wait_tries sets that bound in mbarrier polls (each poll suspends for a bounded,
 * implementation-defined time, about 3.8 us on GB300; 0 restores the default 2^18, about
 * one second).  skip_copies != 0 makes the
 * hop kernels of this context issue no copies, so that nothing completes the barrier and
 * every wait runs out; 0 restores normal operation.  Settings apply to later calls (a CUDA
 * graph captured inside a solve takes them at capture).  Returns DWF_EINVAL for a null ctx. */
dwf_status dwf_debug_set_wait(dwf_ctx *ctx, unsigned wait_tries, int skip_copies);

/* Text of the last error on ctx ("" if none); valid until the next call on ctx. */
const char *dwf_last_error(const dwf_ctx *ctx);
/* Name of a status code. */
const char *dwf_status_string(dwf_status st);

#ifdef __cplusplus
}
#endif
#endif /* DWF_H */
