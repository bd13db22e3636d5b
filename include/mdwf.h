/*
 * libmdwf — even-odd preconditioned Moebius domain-wall fermion solves on one
 * GB300 GPU (sm_103a).
 *
 * The method is the valence-quark solve of arXiv:1701.07559: the Moebius
 * domain-wall operator (Sec. II, kernel (b5+c5) D_W / (2 + (b5-c5) D_W) with
 * domain-wall height M5), applied on gradient-flowed SU(3) links (Sec. III),
 * inverted through the asymmetric even-odd Schur complement (Sec. VII) by a
 * mixed-precision conjugate-gradient solver on the normal equations (Sec. VII,
 * "double-half mixed precision").
 *
 * Operators (DeGrand-Rossi gamma basis, gamma_5 = diag(1,1,-1,-1); periodic in
 * x, y, z; antiperiodic in t unless turned off in mdwf_load_gauge):
 *   H psi(x)  = sum_mu (1 - g_mu) U_mu(x) psi(x+mu) + (1 + g_mu) U_mu(x-mu)^+ psi(x-mu)
 *   D_W       = (4 - M5) - H / 2
 *   (P psi)_s = P_- psi_{s+1} + P_+ psi_{s-1},  psi_{L5} = -m_f psi_0,  psi_{-1} = -m_f psi_{L5-1}
 *   D         = D_W (b5 + c5 P) + (1 - P)          (5D Moebius operator)
 *   Mhat      = A_ee - D_eo A_oo^-1 D_oe,  A = (b5 d + 1) + (c5 d - 1) P,  d = 4 - M5,
 *               D_eo = -1/2 H_eo (b5 + c5 P)
 *
 * Host layouts (FP64, complex interleaved re, im; x fastest):
 *   gauge   U[t][z][y][x][mu][a][b]            mu = 0..3 for x, y, z, t
 *   4D      psi[t][z][y][x][spin][colour]
 *   5D      psi[s][t][z][y][x][spin][colour]   s = 0..L5-1
 *
 * Ownership: the caller owns every buffer passed in; the library copies what
 * it needs (gauge fields are copied to the device at load time) and never
 * frees caller memory.  `_dev` variants take device pointers in the same
 * layouts plus a cudaStream_t (as void*; NULL = the context's own stream) and
 * run asynchronously on that stream, except where noted.
 *
 * Errors: every call returns MDWF_OK (0) or a negative MDWF_ERR_* code;
 * mdwf_last_error(ctx) returns a message for the last failure on ctx.
 * A context is used by one host thread at a time.
 */
#ifndef MDWF_H
#define MDWF_H

#ifdef __cplusplus
extern "C" {
#endif

#define MDWF_OK 0
#define MDWF_ERR_ARG (-1)           /* invalid argument (sizes, ids, null pointers) */
#define MDWF_ERR_NOMEM (-2)         /* device allocation failed */
#define MDWF_ERR_NONFINITE (-3)     /* NaN or Inf in an input */
#define MDWF_ERR_NOT_CONVERGED (-4) /* max_iter reached; outputs hold the best iterate, stats filled */
#define MDWF_ERR_TIMEOUT (-5)       /* a bounded device wait ran out */
#define MDWF_ERR_CUDA (-6)          /* a CUDA runtime call failed */
#define MDWF_ERR_STATE (-7)         /* gauge field or action not set for this cfg_id */
#define MDWF_ERR_FULL (-8)          /* a session has no free slot */

/* Storage precision of the inner (sloppy) solver vectors.  Arithmetic is FP64
 * for MDWF_PREC_DOUBLE and FP32 otherwise; the solution accumulator, the
 * reliable-update residuals and all global sums are FP64 in every mode. */
#define MDWF_PREC_DOUBLE 0
#define MDWF_PREC_SINGLE 1
#define MDWF_PREC_HALF 2 /* fp16 with one float scale per (site, slice, RHS) */
#define MDWF_PREC_BF16 3

typedef struct mdwf_ctx mdwf_ctx;

typedef struct {
  int precision;   /* MDWF_PREC_* (default MDWF_PREC_HALF) */
  int max_iter;    /* CG iterations per RHS (default 100000) */
  double delta;    /* reliable update when |r| < delta * max |r| since the last one (default 0.1) */
  int chunk;       /* CG iterations per device launch sequence between host checks (default 16) */
  int use_graph;   /* capture each chunk in a CUDA graph (default 1) */
  int nsb;         /* half-lattice sites per thread block (0 = chosen by the library) */
  int profile;     /* 1: time every inner-precision hop launch with CUDA events (stats.hop_*) */
  double wait_timeout_s; /* bound of every device-side wait (default 2 s); a wait that runs out ends
                            the call with MDWF_ERR_TIMEOUT and leaves the context usable */
  int timeout_test;      /* testing only: 1 makes each staged-copy wait expect bytes that never
                            arrive, so the bound above must end the call with MDWF_ERR_TIMEOUT */
  int hop_variant;       /* 0: automatic: the autotuner times the CUDA-core direct hop with 1..8
                            sites per block (and, for fp16 storage, form 7 with 1..4) once per (L5, N,
                            precision) and context and keeps the fastest; all of them give identical
                            results.
                            1: CUDA-core hop with direct neighbour loads (FP32 arithmetic: two fifth-
                            dimension slices per thread in packed FP32); 2: CUDA-core hop with
                            neighbours staged in shared memory by bulk copies; 3: tensor-core colour
                            multiply (fp16 storage only, else as 1): thread-per-unit loads when the block
                            is whole warps and L5 x RHS-per-block is a multiple of 8, else 8-unit tiles;
                            4: as 0 with the staged and tensor-core hops among the candidates (their
                            roundings differ from the direct form); 5: tensor-core tiles double-buffered
                            through bulk copies (bounded waits); 6: CUDA-core direct hop, one
                            (site, slice, RHS) unit per thread; 7: as 1, with the block's links in
                            shared memory and each thread's neighbour loads issued two directions
                            ahead by asynchronous copies (fp16 storage with 18-real links, else as 1;
                            the same results as 1) */
  int schur;              /* 0: the asymmetric Schur operator A - D_eo A^-1 D_oe (default, the form
                            Chroma used, Sec. VII); 1: the symmetric form 1 - A^-1 D_eo A^-1 D_oe the
                            paper names as the next step (same x; CUDA-core hops only) */
  int max_restarts;       /* a system whose FP64 full-lattice certificate misses tol resumes from its x
                            with a 16 times tighter Schur stopping norm, at most this often (default 3) */
  double stop_scale_test; /* testing only: multiplies the Schur stopping norm (default 1); above 1 the
                            first certificate misses tol, so the restarts above must finish the solve */
  int link_recon;         /* reals read per link by the inner (FP32-arithmetic) hops: 18 (default) or 12,
                            the first two rows, with the third rebuilt in the kernel as the conjugate
                            cross product (SU(3); the antiperiodic time phase is a separate sign);
                            applies to the default direct hop (hop_variant 0, 1; 7 falls back to 1) */
} mdwf_solver_opts;

typedef struct {
  int iters;             /* CG iterations */
  int reliable_updates;  /* FP64 residual recomputations (including the initial one) */
  int converged;         /* 1 if rel_true_resid <= tol */
  int hop_launches;      /* inner-precision hop launches timed (opts.profile), batch total */
  double rel_true_resid; /* ||b - D x|| / ||b|| of the returned x, in FP64 on the full lattice */
  double time_s;         /* wall time of the call */
  double hop_ms;         /* summed device time of those launches (opts.profile), batch total */
  long long kernel_launches; /* kernels this call put on the GPU, batch total */
  long long hop_units;   /* (site, slice, RHS) units per inner hop launch */
  double phase_ms[5];    /* with opts.profile: device time of the call's phases, batch total:
                            [0] set-up and Schur preparation (source packing, bhat, first residual),
                            [1] CG iterations (graph chunks), [2] FP32 reliable updates,
                            [3] FP64 re-references, [4] reconstruction, FP64 certification, unpacking */
  int fp32_updates;      /* reliable updates with FP32 arithmetic of this system */
  int fp64_rerefs;       /* FP64 re-references of this system (the first residual included) */
  int restarts;          /* resumptions after a missed certificate (opts.max_restarts), batch total */
} mdwf_solve_stats;

/* Fill opts with the defaults listed above. */
void mdwf_default_opts(mdwf_solver_opts* opts);

/* Create a context for lattice dims = {Lx, Ly, Lz, Lt} (each even, >= 2) on CUDA
 * device `device`.  *out receives the context.  Errors: ARG, CUDA, NOMEM. */
int mdwf_create(const int dims[4], int device, mdwf_ctx** out);

/* Release all device memory of ctx and the context itself.  NULL is accepted. */
int mdwf_destroy(mdwf_ctx* ctx);

/* Message of the last error on ctx (never NULL; empty when none). */
const char* mdwf_last_error(const mdwf_ctx* ctx);

/* Copy a gauge field (host, layout above, 18 * 4 * V doubles) into gauge slot
 * cfg_id (>= 0) of ctx, replacing any previous field there.  t_antiperiodic = 1
 * gives the fermion a -1 on hops across the time boundary (the convention of
 * the paper's ensembles), 0 makes time periodic.  Errors: ARG, NONFINITE, NOMEM, CUDA. */
int mdwf_load_gauge(mdwf_ctx* ctx, int cfg_id, const double* U, int t_antiperiodic);

/* Set the Moebius action of cfg_id: domain-wall height M5, Moebius b5, c5
 * (Sec. II), quark mass m_f, fifth-dimension extent L5 (2..32).  The paper's
 * tuned values are in its Table II.  Errors: ARG. */
int mdwf_set_action(mdwf_ctx* ctx, int cfg_id, double M5, double b5, double c5, double mf, int L5);

/* Hopping term on all L5 slices, out = H in (dagger = 0) or H^+ in (dagger = 1),
 * in FP64.  out_parity = 0 or 1 writes the sites of that parity (reading the
 * other parity of `in`) and zeroes the rest of out; -1 writes every site.
 * in, out: host 5D fields of L5 * V * 24 doubles.  Errors: ARG, STATE, NONFINITE, CUDA. */
int mdwf_apply_dslash(mdwf_ctx* ctx, int cfg_id, const double* in, double* out, int out_parity, int dagger);

/* The 5D Moebius operator on the full lattice in FP64: out = D in (dagger = 0)
 * or D^+ in (dagger = 1).  Host 5D fields.  Errors: ARG, STATE, NONFINITE, CUDA. */
int mdwf_apply_mdwf(mdwf_ctx* ctx, int cfg_id, const double* in, double* out, int dagger);

/* The asymmetric Schur operator on even sites (Sec. VII): out_e = Mhat in_e
 * (dagger = 0) or Mhat^+ in_e.  Host 5D full-lattice fields; odd sites of in are
 * ignored and odd sites of out are set to zero.  precision = MDWF_PREC_* selects
 * the storage/arithmetic of the kernels that run (FP64 for MDWF_PREC_DOUBLE).
 * Errors: ARG, STATE, NONFINITE, CUDA. */
int mdwf_apply_schur(mdwf_ctx* ctx, int cfg_id, const double* in, double* out, int dagger, int precision);

/* A fifth-dimension operator on the full lattice in FP64: op = 0 for
 * A = (b5 d + 1) + (c5 d - 1) P, 1 for B = b5 + c5 P, 2 for A^-1 (closed form);
 * dagger = 1 for the adjoint.  Host 5D fields.  Errors: ARG, STATE, CUDA. */
int mdwf_apply_5d(mdwf_ctx* ctx, int cfg_id, int op, const double* in, double* out, int dagger);

/* 5D source from a 4D field eta (host, V * 24 doubles):
 * src = (1 - c5 D_W) (P_+ eta delta_{s,0} + P_- eta delta_{s,L5-1}), the wall
 * injection under which q = P_- x_0 + P_+ x_{L5-1} (mdwf_extract_prop4d) is the
 * 4D quark propagator of the Moebius kernel.  Errors: ARG, STATE, NONFINITE, CUDA. */
int mdwf_make_source(mdwf_ctx* ctx, int cfg_id, const double* eta4d, double* src5d);

/* Solve D x = src for one host 5D source to ||src - D x|| / ||src|| <= tol,
 * through the even-odd Schur complement with CG on the normal equations and
 * reliable updates in FP64.  x5d (host) receives x.  opts may be NULL
 * (defaults); stats may be NULL.  Errors: ARG, STATE, NONFINITE, NOMEM, CUDA,
 * NOT_CONVERGED (x5d holds the last iterate). */
int mdwf_solve(mdwf_ctx* ctx, int cfg_id, const double* src5d, double* x5d, double tol,
               const mdwf_solver_opts* opts, mdwf_solve_stats* stats);

/* Solve n systems in one batched launch sequence: D(m_i) x_i = srcs[i], the
 * action of cfg_id with the quark mass replaced by masses[i] (masses may be NULL
 * for the action's m_f).  srcs[i], xs[i]: host 5D fields; stats: n entries or
 * NULL.  All right-hand sides share every kernel launch; each keeps its own CG
 * scalars and stops on its own.  Errors as mdwf_solve (NOT_CONVERGED if any
 * system did not converge). */
int mdwf_solve_batch(mdwf_ctx* ctx, int cfg_id, int n, const double* const* srcs, const double* masses,
                     double* const* xs, double tol, const mdwf_solver_opts* opts, mdwf_solve_stats* stats);

/* As mdwf_solve_batch with device pointers (layout above) on `stream`.  The
 * call returns when the solves are finished (it reads convergence flags back
 * between chunks).  Errors as mdwf_solve_batch. */
int mdwf_solve_batch_dev(mdwf_ctx* ctx, int cfg_id, int n, const double* const* srcs, const double* masses,
                         double* const* xs, double tol, const mdwf_solver_opts* opts, mdwf_solve_stats* stats,
                         void* stream);

/* The Schur operator of the solver for n right-hand sides at once, on device
 * fields (layout above): out_i = Mhat(m_i) in_i (dagger = 0) or Mhat(m_i)^+ in_i,
 * with m_i = masses[i] (host array; NULL = the action's m_f).  It runs the same
 * kernels, tiling and storage precision (MDWF_PREC_*) as the CG iterations of
 * mdwf_solve_batch; odd sites of in_i are ignored and odd sites of out_i set
 * to zero.  hop_variant as in mdwf_solver_opts in its low 8 bits; bits 8..15, if
 * nonzero, fix the number of sites per thread block (a tuning knob); bit 16 reads
 * 12-real links (opts.link_recon = 12).  Returns
 * after the work on `stream` has finished.
 * Errors: ARG, STATE, NOMEM, CUDA, TIMEOUT. */
int mdwf_apply_schur_batch_dev(mdwf_ctx* ctx, int cfg_id, int n, const double* const* in, double* const* out,
                               const double* masses, int dagger, int precision, int hop_variant, void* stream);

/* mdwf_apply_schur_batch_dev for callers that cannot allocate device memory.
 *
 * Some callers may not call cudaMalloc at all: a host application whose own
 * pool already owns the device memory, or a latency-bound path that cannot
 * accept the device-wide synchronisation an allocation can cause.  This entry
 * point computes the same result as mdwf_apply_schur_batch_dev (same kernels,
 * hop variant 1) but allocates nothing.  Its scratch -- packed copies of the
 * inputs, two intermediate fields, the packed output and the per-RHS masses --
 * lives in one fixed device array of MDWF_NOALLOC_SCRATCH_BYTES bytes that is
 * part of the library's device image: every GPU on which the library's device
 * code is loaded holds those bytes until the process exits.  The caller still
 * allocates and passes the input and output fields.
 *
 * Limit: 4 fields of (V/2) * L5 * n stored spinors (192, 96, 48 or 48 bytes each
 * for double, single, half, bf16, plus a 4-byte scale each for half) plus the
 * masses must fit, e.g. FP64 up to about 87,000 (site, slice, RHS) units.  A
 * larger problem is rejected with MDWF_ERR_ARG and a message giving the size.
 *
 * The call is synchronous: it copies the masses from host memory and returns
 * when its work on `stream` has finished, so it cannot be captured in a CUDA
 * graph.  It looks up the array's device address on every call (no cached
 * address survives a device reset).  Every call uses the same array, which
 * keeps the previous call's
 * contents (the kernels overwrite what they read, and the one field that must
 * start at zero is cleared by the call itself); calls that overlap on the GPU --
 * from several streams or host threads at once -- race on the array and must be
 * serialised by the caller.  The paper has no counterpart to this entry point.
 * Errors: ARG (including a problem too large for the array), STATE, CUDA. */
#define MDWF_NOALLOC_SCRATCH_BYTES (64u * 1024u * 1024u)
int mdwf_apply_schur_batch_dev_noalloc(mdwf_ctx* ctx, int cfg_id, int n, const double* const* in,
                                       double* const* out, const double* masses, int dagger, int precision,
                                       void* stream);

/* Device-pointer variants of the operator applies, on `stream` (asynchronous). */
int mdwf_apply_dslash_dev(mdwf_ctx* ctx, int cfg_id, const double* in, double* out, int out_parity, int dagger,
                          void* stream);
int mdwf_apply_mdwf_dev(mdwf_ctx* ctx, int cfg_id, const double* in, double* out, int dagger, void* stream);

/* ---- Domain decomposition in time -----------------------------------------
 * A lattice split along t into P sub-domains (multi-GPU mode of the paper's
 * runs, Sec. VII, Table VII geometries 1.1.1.P): each sub-domain is a context
 * of dims {Lx, Ly, Lz, Lt/P} (Lt/P even, so local and global parities agree)
 * holding every L5 slice of its sites and the links of its slab.  A hop across
 * the slab's time edges reads the neighbouring sub-domain's face, 12 reals per
 * (3D site, slice): the next sub-domain's first slice projected as the forward
 * hop projects it, and the previous sub-domain's last slice projected and
 * multiplied by U_t^+ with the sender's own links, so no link crosses a
 * boundary.  Faces are laid out [z][y][x][s][spin 2][colour 3][re, im]
 * (Lx Ly Lz L5 12 doubles), device memory owned by the caller; the caller moves
 * them between sub-domains (a device copy, or a send into the receiving GPU's
 * own buffer).  FP64, one right-hand side, the API field layout (device).
 *
 * mdwf_dd_pack_faces_dev: the faces of the field the hop of `kind` reads
 * (kind 0: in, for out = H in or H^+ in; kind 1: B in for D (dagger 0), in for
 * D^+): face_prev gets the first slice (for the previous sub-domain),
 * face_next the last slice (for the next one).  `dagger` as in the apply.
 * mdwf_dd_apply_dev: out = H in, H^+ in (kind 0) or D in, D^+ in (kind 1) on
 * the sub-domain, the time hops across its edges taken from halo_next (the
 * next sub-domain's face_prev) and halo_prev (the previous one's face_next),
 * each multiplied by its sign (-1 across the global antiperiodic time
 * boundary, else 1; the context's own boundary flag is not used).  Both
 * return after the work on `stream` has finished.  The result equals the
 * undecomposed operator bit for bit (same operations in the same order).
 * Errors: ARG (odd local time extent, bad kind, null pointer), STATE, CUDA. */
int mdwf_dd_pack_faces_dev(mdwf_ctx* ctx, int cfg_id, int kind, int dagger, const double* in, double* face_prev,
                           double* face_next, void* stream);
int mdwf_dd_apply_dev(mdwf_ctx* ctx, int cfg_id, int kind, int dagger, const double* in, double* out,
                      const double* halo_next, const double* halo_prev, double sign_next, double sign_prev,
                      void* stream);

/* ---- Solver sessions: continuous batching --------------------------------
 * A session keeps the device state of `slots` right-hand sides of one gauge
 * configuration resident.  Requests (a 5D source, a quark mass, an output field,
 * a caller tag) enter free slots between CG chunks; every chunk advances all
 * occupied slots in the same kernel launches; converged slots are reconstructed,
 * checked in FP64 and written to their output field, and become free again.
 * This is the serving loop of the batched solve (the paper's propagator solves,
 * Sec. VII, as requests); a request gives the same x alone as in any mix.
 * All pointers are device fields in the API layout; calls on one session come
 * from one host thread.  Sessions of different contexts run on their own
 * streams and overlap on the device. */
typedef struct mdwf_session mdwf_session;

/* Device bytes a session of `slots` slots holds (for admission control), or -1. */
long long mdwf_session_bytes(mdwf_ctx* ctx, int cfg_id, int slots, int precision);

/* Create a session on `stream` (NULL: the context's stream) with the solver
 * options (precision, delta, chunk, max_iter, ...) and tolerance of every solve.
 * Errors: ARG, STATE, NOMEM, CUDA. */
int mdwf_session_create(mdwf_ctx* ctx, int cfg_id, int slots, const mdwf_solver_opts* opts, double tol, void* stream,
                        mdwf_session** out);
int mdwf_session_destroy(mdwf_session* s);

/* Put a request into a free slot (returned in *slot): source src5d (read now),
 * quark mass, solution field x5d (written when the request completes), tag.
 * Errors: FULL (no free slot), ARG, NONFINITE, CUDA. */
int mdwf_session_submit(mdwf_session* s, const double* src5d, double mass, double* x5d, long long tag, int* slot);

/* Enqueue `iters` CG iterations (0: opts.chunk) of every occupied slot on the
 * session's stream and return without waiting. */
int mdwf_session_launch(mdwf_session* s, int iters);

/* Wait for the session's work, run its reliable updates, and complete up to
 * max_done converged slots (tags[] and stats[] receive them, *n_done their number;
 * stats.time_s is the time since submit).  Errors: CUDA, TIMEOUT. */
int mdwf_session_poll(mdwf_session* s, int max_done, long long* tags, mdwf_solve_stats* stats, int* n_done);

/* Number of occupied slots. */
int mdwf_session_occupied(const mdwf_session* s);

/* mdwf_make_source on device fields (eta4d: V * 24 doubles; src5d: L5 * V * 24), on `stream`. */
int mdwf_make_source_dev(mdwf_ctx* ctx, int cfg_id, const double* eta4d, double* src5d, void* stream);

/* Residual-mass correlators (Eq. mres, Sec. III): for the n 5D solutions xs
 * (device, API layout; the solves of point sources, one per source spin and
 * colour), per time slice t (host arrays of Lt doubles)
 *   c_pp[t]  = sum_{x in t, sources, spin, colour} |q(x)|^2,  q = P_- x_0 + P_+ x_{L5-1}
 *   c_j5q[t] = the same for Q = P_+ x_{L5/2-1} + P_- x_{L5/2} (the midpoint field),
 * P_+- = (1 +- gamma_5) / 2.  With the sources of mdwf_make_source these are the
 * pseudoscalar and midpoint-pseudoscalar correlators of the paper's ratio, and
 * m_res(t) = c_j5q[t] / c_pp[t].  FP64, fixed summation order.  Errors: ARG,
 * STATE, NOMEM, CUDA. */
int mdwf_mres_correlators_dev(mdwf_ctx* ctx, int cfg_id, int n, double* const* xs, double* c_pp, double* c_j5q,
                              void* stream);

/* The autotuner on its own: the inner hop form and sites per block that the
 * solver uses for n right-hand sides of this configuration at `precision`
 * (include_tensor_core: also try the tensor-core hop), with its time for one
 * Mhat + Mhat^+ application.  Runs the timing once per (L5, n, precision,
 * candidate set) and context, then answers from the cache.  The timing runs use
 * (and leave allocated) the context's solver workspace for n RHS, the fields a
 * solve of n RHS would use.  Outputs may be NULL.
 * Errors: ARG, STATE, NOMEM, CUDA, TIMEOUT. */
int mdwf_autotune(mdwf_ctx* ctx, int cfg_id, int n, int precision, int include_tensor_core, int* hop_variant,
                  int* nsb, double* ms_per_pair);

/* Wilson (gradient) flow of a gauge field on the device, in place: U is a
 * device array in the mdwf_load_gauge layout (V * 4 * 18 doubles) of this
 * context's lattice; nsteps steps of size eps of Luscher's three-stage
 * Runge-Kutta scheme for dV/dt = -P_TA(Omega) V (Wilson plaquette action), in
 * FP64 (the smoothing of Sec. III, flow time nsteps * eps).  Input preparation:
 * load the result with mdwf_load_gauge.  Holds 3 * 4V * 18 doubles of scratch
 * during the call.  Errors: ARG, NOMEM, CUDA. */
int mdwf_wilson_flow_dev(mdwf_ctx* ctx, double* U, double eps, int nsteps, void* stream);

/* Average plaquette (1/(18 V)) sum_{x, mu<nu} Re tr P_mu_nu(x) of a device gauge
 * field U (layout as above); synchronous, result in *plaq (host). */
int mdwf_plaquette_dev(mdwf_ctx* ctx, const double* U, double* plaq);

/* Gauge-covariant Gaussian smearing of a 4D source in place (device field eta4d,
 * V * 24 doubles, the mdwf_make_source layout): n_iter steps of
 *   eta <- eta + k sum_{i=x,y,z} [U_i(x) eta(x+i) + U_i(x-i)^+ eta(x-i) - 2 eta(x)],
 * k = sigma^2 / (4 n_iter), on the links of cfg_id (which tends to
 * exp(sigma^2 Delta / 4) eta; a point source spreads to variance sigma^2 / 2 per
 * direction).  The paper's propagators use gauge-covariant Gaussian-smeared
 * sources (Sec. VII); it does not give the width.  FP64.  Errors: ARG, STATE, NOMEM, CUDA. */
int mdwf_smear_source_dev(mdwf_ctx* ctx, int cfg_id, double* eta4d, double sigma, int n_iter, void* stream);

/* Z2 noise 4D source on a device field eta4d (V * 24 doubles), on `stream`:
 * complex element k ([t][z][y][x][spin][colour] order) is +1 or -1 (imaginary
 * part 0) by the top bit of the k-th output of SplitMix64 started from `seed`
 * (Steele, Lea and Flood, OOPSLA 2014).  A synthetic input for serving
 * workloads; the paper's own sources (Sec. III) are smeared point sources. */
int mdwf_z2_source_dev(mdwf_ctx* ctx, unsigned long long seed, double* eta4d, void* stream);

/* 4D propagator from a 5D solution: q = P_- x_0 + P_+ x_{L5-1} (host arrays;
 * x5d has L5 * V * 24 doubles, q4d V * 24).  Pure host code.  Errors: ARG. */
int mdwf_extract_prop4d(const double* x5d, const int dims[4], int L5, double* q4d);

#ifdef __cplusplus
}
#endif
#endif /* MDWF_H */
