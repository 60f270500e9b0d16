/*
 * aim.h - C ABI of the GB300 library for the numerically filtered Adaptive Integral Method
 * (AIM) applied to the 2-D electric field integral equation (EFIE).
 *
 * Method: T. Pignatelli, V. Giunzioni, P. Ricci, M. E. Masciocchi, A. Merlini,
 * F. P. Andriulli, "A Numerical Approach to Operator Filtering within the Adaptive
 * Integral Method for Electromagnetic Integral Equations".
 *
 * What the library computes (section / equation of that paper):
 *   - TE-EFIE operators on a closed curve with piecewise-linear hats and Galerkin testing
 *     (Sec. II, Eqs. 1-4): the single layer S, the hypersingular N, the Gram matrix G,
 *     and the Calderon-preconditioned operator G^-1 S G^-1 N (Eq. 3);
 *   - their AIM matrix-vector products (Sec. III-A, Eqs. 7-8): projection of the
 *     quadrature nodes onto a uniform m x m grid, circulant embedding of the grid kernel,
 *     an FFT product, and interpolation back;
 *   - the numerically filtered S^alpha (Sec. III-B, Eq. 10): the kernel spectrum F(c_grid)
 *     truncated to the disc |kappa| <= alpha, with the grid self term set to zero
 *     (Sec. III-C);
 *   - the TM-EFIE (pulse basis, midpoint collocation) single-layer system on the same
 *     grid machinery, filtered or not;
 *   - GMRES solves of these systems (the paper's "iterative solvers", Sec. I).
 * Unfiltered operators carry a sparse near-field correction (exact singular quadrature
 * minus the AIM entry for close pairs); the paper itself only zeroes the grid self term.
 *
 * Conventions
 *   - Lengths and the wavenumber k share one unit; time dependence e^{+j w t};
 *     g(r) = -(j/4) H0^(2)(k r); eta = 1.
 *   - Complex vectors are interleaved (re, im) complex128 in every precision mode; the mode
 *     (AIM_FP64, AIM_MIXED, AIM_FP64_NATIVE, below) selects the grid arithmetic only.
 *   - Multi-vector arguments are column-major: vector r of nrhs starts at element r*n.
 *   - Vector pointers may be device memory or host memory (pageable or pinned); the
 *     library detects which (cudaPointerGetAttributes) and stages host data through
 *     its own device buffers on the call's stream. The caller keeps ownership.
 *   - `stream` is a cudaStream_t (NULL: the legacy default stream). Calls return after
 *     enqueueing device work unless stated otherwise; results in host memory are
 *     complete when the call returns.
 *   - Every entry point returns a status; none exits, traps or aborts. A one-line reason
 *     for the last failure on the calling thread is returned by aim_last_error().
 *   - Calls on one context must not overlap (no internal locking); different contexts may
 *     be used concurrently from different threads and streams.
 *   - A context lives on the CUDA device that was current at aim_setup. Every call that
 *     enqueues work on it returns AIM_EINVAL, before any launch, when another device is
 *     current on the calling thread.
 */
#ifndef AIM_GB300_H
#define AIM_GB300_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  AIM_OK = 0,
  AIM_EINVAL = 1,    /* an argument is out of range or inconsistent */
  AIM_ENOMEM = 2,    /* a device or host allocation failed, or a memory budget was exceeded */
  AIM_ECUDA = 3,     /* a CUDA runtime call failed */
  AIM_ENOCONV = 4,   /* GMRES reached max_iter without meeting the tolerance */
  AIM_ENUMERIC = 5,  /* a non-finite value appeared (NaN/Inf in inputs or residuals) */
  AIM_ETIMEOUT = 6,  /* the solve exceeded its time limit */
  AIM_ESTATE = 7     /* the call does not apply to this context (e.g. TE operator on a TM context) */
} aim_status;

typedef enum {
  AIM_TM_PULSE_COLLOC = 0,  /* TM-EFIE: pulse basis per segment, collocation at segment midpoints */
  AIM_TE_P1_GALERKIN = 1    /* TE-EFIE: P1 hat per vertex, Galerkin testing (Sec. II) */
} aim_form;

typedef enum {
  AIM_OP_S = 0,               /* single layer S (Eq. 4): AIM + near-field correction */
  AIM_OP_S_ALPHA = 1,         /* numerically filtered S^alpha (Eq. 10), no correction */
  AIM_OP_N = 2,               /* TE only: hypersingular N (Eq. 2) in Maue form, AIM + near field */
  AIM_OP_CALDERON = 3,        /* TE only: G^-1 S G^-1 N (Eq. 3) */
  AIM_OP_CALDERON_ALPHA = 4,  /* TE only: G^-1 S^alpha G^-1 N (Eq. 3 with Eq. 10) */
  AIM_OP_GRAM_INV = 5,        /* TE only: G^-1 (G of Eq. 3) */
  AIM_OP_EFIE = 6,            /* system matrix of the EFIE: TM j k eta S ; TE N (Eq. 1 scaled by jk/eta) */
  AIM_OP_EFIE_ALPHA = 7,      /* TM only: j k eta S^alpha */
  AIM_OP_N_ALPHA = 8,         /* TE only: N with the filtered kernel of Eq. 10 in all three
                                 projections, no near-field correction */
  AIM_OP_CALDERON_ALPHA2 = 9  /* TE only: G^-1 S^alpha G^-1 N^alpha (Eq. 3, both operators filtered) */
} aim_op;

/* Grid arithmetic of a product (vectors are complex128 in every mode):
 *   AIM_FP64        FP64-accurate (relative rounding ~2^-48 per operation): double-float
 *                   arithmetic on the FP32 pipe, since GB300's FP64 pipe is ~1/64 of its FP32
 *                   pipe; grid intermediates are 16 bytes per complex.
 *   AIM_MIXED       complex64 grid products and interpolation sums (FP32 arithmetic); near-field
 *                   values stored as complex64 and applied with FP64 sums.
 *   AIM_FP64_NATIVE IEEE binary64 grid arithmetic on the FP64 pipe (the reference the other
 *                   two are tested against). */
enum { AIM_FP64 = 0, AIM_MIXED = 1, AIM_FP64_NATIVE = 2 };

/* Geometry: a closed polygon, counter-clockwise, given by its n_seg vertices (x0,y0,x1,y1,...).
 * Segment e joins vertex e to vertex e+1 (mod n_seg). The unknowns are one per segment (TM)
 * or one per vertex (TE); either way there are n_seg of them. */
typedef struct {
  int n_seg;
  const double* xy;   /* host pointer, 2*n_seg doubles; copied by aim_setup */
  aim_form form;
  int quad_p;         /* Gauss-Legendre nodes per segment used by the projections (Eq. 7), 1..16 */
} aim_geometry;

/* Grid (Sec. III-A): m points per side spanning [-L, L]^2, spacing eps = 2L/(m-1).
 * half_side_L <= 0 selects L = R/(1-(s+2)/(m-1)), R = max |vertex coordinate|.
 * fft_P is the circulant embedding side: 0 selects the smallest power of two >= max(2m-1, 64);
 * otherwise it must be a power of two with max(2m-1, 64) <= fft_P <= 4096. */
typedef struct {
  int m;
  double half_side_L;
  int fft_P;
} aim_grid;

/* Interpolation stencil: s points per axis (Lagrange, 2..12); near_radius <= 0 selects s*eps.
 * Hat (or segment) pairs whose supports come within near_radius get exact entries in the
 * unfiltered operators. */
typedef struct {
  int s;
  double near_radius;
} aim_stencil;

/* Filter of the "alpha" operators (S^alpha, N^alpha, the filtered Calderon products, the TM
 * filtered EFIE); requires alpha > k. `enabled` selects how the filtered kernel is made:
 *   AIM_FILTER_NONE       no filter: the alpha operators equal the unfiltered ones without their
 *                         near-field correction;
 *   AIM_FILTER_NUMERICAL  the paper's numerical filter (Sec. III-B, Eq. 10): the spectrum of the
 *                         grid kernel F(c_grid), self term zeroed (Sec. III-C), truncated to the
 *                         disc kappa <= alpha, kappa = 2 pi sqrt(p~^2 + q~^2)/(P eps);
 *   AIM_FILTER_ANALYTIC   the analytically filtered kernel g^alpha of Eq. 6 sampled at the grid
 *                         offsets, g^alpha(eps sqrt(i~^2 + j~^2)), and transformed: the AIM form of
 *                         the analytic filter the paper compares with (Fig. 1a, Figs. 2-3). Its
 *                         samples cost a principal-value integral each (FP64, about alpha r / 8
 *                         panels of 20 nodes at distance r); setup time grows like P^3. */
enum { AIM_FILTER_NONE = 0, AIM_FILTER_NUMERICAL = 1, AIM_FILTER_ANALYTIC = 2 };
typedef struct {
  int enabled;
  double alpha;
} aim_filter;

typedef struct {
  double tol;          /* relative residual target ||b - A x|| / ||b|| of the solved system */
  int restart;         /* GMRES restart length (1..10000); the Krylov basis takes
                          (restart+4) * n * nrhs * 16 bytes of device memory and the
                          Hessenberg matrix about restart^2/2 * nrhs * 16 bytes */
  int max_iter;        /* total inner iterations per right-hand side */
  int precision;       /* AIM_FP64, AIM_FP64_NATIVE, or AIM_MIXED (FP32 grid inner solves inside
                          iterative refinement with AIM_FP64 residuals) */
  double inner_tol;    /* mixed only: tolerance of each inner FP32-grid solve, on its Arnoldi residual
                          estimate relative to ||r|| (one Krylov cycle of at most `restart`
                          iterations); <= 0 asks for half the remaining reduction, 0.5 tol ||b||/||r|| */
  int timeout_ms;      /* <= 0: no limit */
} aim_solve_opts;

typedef struct {
  int iters;           /* GMRES iterations (inner iterations summed over refinement steps) */
  int outer_iters;     /* refinement steps (1 in FP64 mode) */
  double rel_res;      /* final relative residual of the solved system, FP64 matvec */
  int converged;       /* 1 if rel_res <= tol */
} aim_solve_info;

typedef struct {
  int n;               /* unknowns */
  int m, fft_P, s, quad_p;
  double k, L, eps, alpha;
  int n_active;        /* grid points touched by the projections */
  int row_lo, row_hi;  /* grid rows holding active points */
  long long nnz_near;  /* near-field correction entries */
  size_t device_bytes; /* device memory held by the context */
  double setup_seconds;
  int filter_kind;     /* AIM_FILTER_NONE, AIM_FILTER_NUMERICAL or AIM_FILTER_ANALYTIC */
} aim_info;

typedef struct aim_ctx aim_ctx;

/* Builds every operator of the context on the current CUDA device (Secs. II-III):
 * quadrature nodes and hat values (Eq. 7), the grid and the projections P = Lambda W Phi
 * (Sec. III-A), the grid kernel samples with the self term set to zero (Sec. III-C), its
 * spectrum and the filtered spectrum (Sec. III-B), the near-field correction, and G.
 * All inputs are host memory and are copied. Work runs on `stream`; the call
 * synchronises it before returning. On success *out owns all device state until
 * aim_destroy. Errors: AIM_EINVAL (n_seg < 3, m < 8, bad P, alpha <= k when enabled,
 * s outside 2..12, quad_p outside 1..16, k <= 0, a vertex outside the grid),
 * AIM_ENOMEM, AIM_ECUDA. */
aim_status aim_setup(const aim_geometry* geometry, double k, const aim_grid* grid,
                     const aim_stencil* stencil, const aim_filter* filter, void* stream,
                     aim_ctx** out);

/* Releases everything the context owns. NULL is allowed. */
void aim_destroy(aim_ctx* ctx);

/* Setup artefacts, saved and reloaded (no counterpart in the paper: a restarted process reloads
 * them instead of recomputing them). A setup blob holds what aim_setup computes: the active grid
 * set and the projections P = Lambda W Phi (Sec. III-A, Eq. 7), the twiddles, G^-1 (Eq. 3), the
 * near-field correction, and the kernel spectrum and filtered spectrum (Sec. III-B, Eq. 10) in
 * FP64. Their complex64 and double-float copies are derived again on import, exactly as aim_setup
 * derives them, so a context made by aim_import_setup gives bit-identical results.
 *
 * aim_setup_key: a 64-bit key (FNV-1a) of everything aim_setup's result depends on: the form,
 * the vertices, k, the derived grid (m, P, L, eps), s, quad_p, the near radius and the filter.
 * Two calls whose arguments describe the same problem (e.g. fft_P = 0 and the P it selects) get
 * the same key. Host only: no CUDA call. Errors: those of aim_setup's argument checks.
 *
 * aim_export_setup: with buf == NULL, sets *bytes to the blob's size. Otherwise *bytes is the
 * size of the host buffer `buf` (AIM_EINVAL if smaller than the blob) and receives the size
 * written. The blob is a 160-byte header (magic "AIMSETUP", format version, key, problem
 * parameters, array counts, a checksum of the payload) followed by the arrays, each starting
 * at a 16-byte offset, little-endian. Copies run on `stream`; the call synchronises it. The
 * caller owns `buf`.
 *
 * aim_import_setup: a context equal to aim_setup(geometry, k, grid, stencil, filter, ...) from a
 * blob that aim_export_setup wrote for that problem. Before any CUDA call it checks the magic,
 * the version, the size, the checksum, every problem parameter and vertex against the
 * arguments, and every index of the stored sparse patterns against its range: AIM_EINVAL
 * (with the reason in aim_last_error) if any differs, so a blob of another problem, a stale
 * format or a corrupted file is refused and never reaches the device. `blob` is host memory,
 * read only during the call. Then as aim_setup: AIM_ENOMEM, AIM_ECUDA; on success *out owns
 * its device state until aim_destroy. */
aim_status aim_setup_key(const aim_geometry* geometry, double k, const aim_grid* grid,
                         const aim_stencil* stencil, const aim_filter* filter,
                         unsigned long long* key);
aim_status aim_export_setup(const aim_ctx* ctx, void* buf, size_t* bytes, void* stream);
aim_status aim_import_setup(const aim_geometry* geometry, double k, const aim_grid* grid,
                            const aim_stencil* stencil, const aim_filter* filter, const void* blob,
                            size_t bytes, void* stream, aim_ctx** out);

aim_status aim_get_info(const aim_ctx* ctx, aim_info* info);

/* Pre-allocates workspaces for up to nrhs simultaneous vectors in the given precision,
 * so that later calls (and CUDA-graph capture of them) allocate nothing. */
aim_status aim_reserve(aim_ctx* ctx, int nrhs, int precision);

/* Launch schedule of the three grid kernels for one precision (no counterpart in the
 * paper). transforms_per_thread: 1 puts the even- and odd-half transforms of a line in
 * adjacent lanes, 2 puts both in one thread (native FP64 allows 2 only). row_threads: the
 * least threads of a row-pass CTA (32..1024; rows are added to a CTA until it has that many).
 * col_cols: columns of one column-pass CTA, a power of two, 0 for the default (the fewest
 * whole 32-byte column tiles that give 128 threads). elems_per_thread: 16 (radix-16 passes)
 * or 8 (radix-8 passes, half the registers per thread; not for native FP64); 0 means 16.
 * Results are identical under every schedule with the same elems_per_thread: the arithmetic
 * and its order do not depend on the rest; the two pass geometries differ by rounding. */
typedef struct {
  int transforms_per_thread;
  int row_threads;
  int col_cols;
  int elems_per_thread;
} aim_schedule;

/* Sets the schedule of `precision` for this context. AIM_EINVAL when it cannot be launched
 * for the context's transform length (launch bound or 227 KB shared-memory limit). */
aim_status aim_set_schedule(aim_ctx* ctx, int precision, const aim_schedule* schedule);
aim_status aim_get_schedule(const aim_ctx* ctx, int precision, aim_schedule* schedule);

/* Autotuner (no counterpart in the paper; a launch-schedule choice). Times the filtered
 * product (S^alpha) for nrhs vectors under each feasible schedule - 16 or 8 elements and one
 * or two transforms per thread, 128, 256 or 1024 row-pass threads, 1 to 8 columns per column-pass
 * CTA - and
 * keeps the fastest for this context and precision. Synchronises `stream`. *chosen (host,
 * may be NULL) receives the winner. */
aim_status aim_autotune(aim_ctx* ctx, int nrhs, int precision, void* stream, aim_schedule* chosen);

/* Right-hand sides for unit plane waves exp(-j k khat.r), khat = (cos th, sin th):
 * TE: E_i = <phi_i, (jk/eta) E_t> with E^i = eta H^i_z (z x khat) (Sec. II, below Eq. 2);
 * TM: E_i = E^i_z(midpoint_i). `angles` is a host array of nrhs angles (radians);
 * `rhs` receives n*nrhs complex128 values (host or device). */
aim_status aim_rhs_planewave(aim_ctx* ctx, int nrhs, const double* angles, void* rhs, void* stream);

/* y = A x for nrhs vectors (complex128 in and out, n*nrhs each; host or device; x and y
 * must not overlap). A is selected by `op` (see aim_op); precision selects the grid
 * arithmetic. The work is the pipeline of Eq. 8 / Eq. 10: sparse anterpolation fused
 * into a forward row FFT, a column FFT fused with the spectral product and the inverse
 * column FFT, an inverse row FFT with restriction, and the interpolation gather fused
 * with the near-field SpMV. Errors: AIM_EINVAL, AIM_ESTATE, AIM_ENOMEM, AIM_ECUDA. */
aim_status aim_matvec(aim_ctx* ctx, aim_op op, int nrhs, const void* x, void* y,
                      int precision, void* stream);

/* y_i = A_i x_i for `count` (1..32) contexts of any sizes at once (no counterpart in the paper; a
 * batching of Eq. 8 / Eq. 10 across problems). Every grid pass stage of all the contexts - the
 * forward row passes with anterpolation, the column passes, the inverse row passes and the
 * gathers with their near-field rows - runs in ONE persistent cooperative launch whose CTAs take
 * work items (context, channel, group of rows or columns) from all of them; the Calderon products
 * take two such launches with the Gram inverses between them (Eq. 3). The launch separates its
 * phases by grid barriers whose waits are bounded (AIM_ETIMEOUT if one gives up). Each result is
 * bit-identical to aim_matvec on that context alone with the same schedule. ctxs, ops, nrhs, x,
 * y: host arrays of `count` entries; x[i], y[i]: device pointers to nrhs[i] vectors of context i;
 * a context appears at most once. All contexts must be current on this device and share the pass
 * geometry (transforms and elements per thread) of their schedule in `precision` (otherwise
 * AIM_EINVAL). One launch serves contexts whose transforms fit one CTA size (a CTA takes
 * max(2, 32-byte tile) lines of the longest transform and correspondingly more lines of shorter
 * ones, at most a context's P); a stage whose contexts span more than that (for example P = 64
 * beside P = 2048) is split into the fewest such launches. Synchronises `stream`. */
aim_status aim_matvec_multi(int count, aim_ctx* const* ctxs, const aim_op* ops, const int* nrhs,
                            const void* const* x, void* const* y, int precision, void* stream);

/* The grid product alone (the bracket of Eq. 8, or of Eq. 10 when filtered != 0) on
 * full m x m grids: v = [F^-1(F(c) .* F(b))]_restr with b = u zero-padded to P x P.
 * u and v hold nrhs row-major m x m complex128 grids (element (iy, ix) at iy*m + ix);
 * host or device. Rows of u outside the context's active row range must be zero; rows of
 * v outside it are returned as zero. */
aim_status aim_grid_product(aim_ctx* ctx, int filtered, int nrhs, const void* u, void* v,
                            int precision, void* stream);

/* Grid kernel tables, for comparing the numerical filter with the analytic one (Sec. III-B,
 * Fig. 1). Each table is the (H+1) x (H+1) quarter, H = fft_P/2, of an array that is even in both
 * indices, written row-major as complex128 (element [a][b] at a*(H+1) + b; host or device `out`).
 *   AIM_TABLE_SPECTRUM            F(c_grid)[p][q]: the DFT of the grid kernel samples
 *                                 g(eps sqrt(i~^2 + j~^2)) with the self term set to zero
 *                                 (Sec. III-A, III-C), as the unfiltered products use it;
 *   AIM_TABLE_SPECTRUM_FILTERED   the spectrum the filtered products use: F(c_grid) truncated to
 *                                 kappa <= alpha (Eq. 10), or the analytic one (AIM_FILTER_ANALYTIC);
 *   AIM_TABLE_ANALYTIC_SAMPLES    g^alpha(eps sqrt(i^2 + j^2)) of Eq. 6 at offset [i][j] (computed
 *                                 on the call's stream; needs a context set up with a filter);
 *   AIM_TABLE_ANALYTIC_SPECTRUM   the DFT of those samples (Fig. 1a; computed likewise).
 * The call synchronises `stream`. Errors: AIM_EINVAL (unknown table, null pointer), AIM_ESTATE
 * (analytic tables of a context without a filter radius), AIM_ENOMEM, AIM_ECUDA. */
enum { AIM_TABLE_SPECTRUM = 0, AIM_TABLE_SPECTRUM_FILTERED = 1, AIM_TABLE_ANALYTIC_SAMPLES = 2,
       AIM_TABLE_ANALYTIC_SPECTRUM = 3 };
aim_status aim_kernel_table(aim_ctx* ctx, int which, void* out, void* stream);

/* Size of the scratch array behind aim_grid_product_noalloc (bytes). */
#define AIM_NOALLOC_SCRATCH_BYTES ((size_t)16 << 20)

/* The grid product of aim_grid_product without any allocation. This entry point has no
 * counterpart in the paper. It is for callers that cannot allocate device memory at the moment
 * they need a product: real-time loops whose device memory is fixed before they start (an
 * allocation there can stall or fail), hosts that forbid cudaMalloc after start-up, and code
 * running inside another runtime's memory pool that third-party libraries may not grow.
 * aim_grid_product may grow the context's workspace with cudaMalloc the first time it sees a
 * larger batch; this variant instead keeps its scratch (the tiled intermediate grid) in a fixed
 * array of AIM_NOALLOC_SCRATCH_BYTES compiled into the library's device image. Every GPU that
 * loads the library holds that array until the process exits. The call makes no cudaMalloc,
 * cudaFree or other allocating call.
 * Same result as aim_grid_product with the same arguments, bit for bit. u and v must be device
 * pointers on the context's device, which must be current.
 * The first call on each device looks up the array's device address (cudaGetSymbolAddress,
 * once per device, under a lock); make that first call before any stream capture.
 * Every call shares the one array and leaves its contents there; nothing in it needs to start at
 * zero (each product writes all of the scratch it later reads). Calls that overlap on the GPU -
 * from any context, stream or thread - race on the array; the caller must serialise them.
 * Errors: AIM_EINVAL if the intermediate grid (nrhs * fft_P * active rows * 16 bytes, 8 in
 * AIM_MIXED) exceeds AIM_NOALLOC_SCRATCH_BYTES, u or v is not device memory, or the current
 * device is not the context's; AIM_ESTATE while kernel timing (aim_profile_start) is active,
 * because timing creates events. */
aim_status aim_grid_product_noalloc(aim_ctx* ctx, int filtered, int nrhs, const void* u, void* v,
                                    int precision, void* stream);

/* Solves A x = b for nrhs right-hand sides by restarted GMRES with FP64 Arnoldi
 * (classical Gram-Schmidt applied twice, the second pass delayed by one step: two reads of the
 * Krylov basis per iteration). `system` is AIM_OP_EFIE, AIM_OP_EFIE_ALPHA,
 * AIM_OP_CALDERON, AIM_OP_CALDERON_ALPHA or AIM_OP_CALDERON_ALPHA2. For the Calderon systems `rhs` is the EFIE
 * excitation E and the solver forms G^-1 S G^-1 E itself (Eq. 3). In AIM_MIXED precision
 * the inner GMRES uses the FP32 grid product and the outer loop refines with FP64
 * residuals until opts->tol. x is both the initial guess (if x0_given != 0) and the
 * result. info receives nrhs entries (host pointer, may be NULL).
 * Returns AIM_ENOCONV, AIM_ETIMEOUT or AIM_ENUMERIC when any right-hand side fails. */
aim_status aim_solve(aim_ctx* ctx, aim_op system, int nrhs, const void* rhs, void* x,
                     int x0_given, const aim_solve_opts* opts, aim_solve_info* info,
                     void* stream);

/* Golub-Kahan-Lanczos bidiagonalisation of an operator, for the singular-value studies of
 * Sec. IV (Figs. 2-3). k steps of
 *     A v_j = alpha_j u_j + beta_{j-1} u_{j-1},   A^H u_j = alpha_j v_j + beta_j v_{j+1},
 * started from v_0 = v0/||v0|| (n complex128, host or device; the caller supplies the start, for
 * instance a seeded random vector), with both bases reorthogonalised in full (classical
 * Gram-Schmidt twice, FP64) and every product A x, A^H x computed by the library's grid product in
 * `precision`. The singular values of the k x k upper bidiagonal matrix with alpha_0..alpha_{k-1} on
 * the diagonal and beta_0..beta_{k-2} above it approximate those of A, and equal them for k = n (up to
 * rounding). alpha, beta: host arrays of k doubles (beta_{k-1} is the norm of the next residual).
 * U (k x n) and V ((k+1) x n): device arrays that receive the Lanczos vectors u_j, v_j row by row, or
 * NULL. The adjoint uses the complex symmetry of the TE Galerkin operators: op is AIM_OP_S, S_ALPHA,
 * N, N_ALPHA, GRAM_INV, EFIE or one of the Calderon products (transposed as the reversed chain
 * N G^-1 S G^-1). Errors: AIM_EINVAL (k < 1 or k > n, another operator, U/V not device memory),
 * AIM_ESTATE (TM context: collocation operators are not symmetric), AIM_ENUMERIC, AIM_ENOMEM,
 * AIM_ECUDA. Synchronises `stream`. */
aim_status aim_lanczos_bidiag(aim_ctx* ctx, aim_op op, int k, int precision, const void* v0,
                              double* alpha, double* beta, void* U, void* V, void* stream);

/* Fused products of concurrent solves (no counterpart in the paper; the batching side of serving).
 * A batcher is shared by solves that run at the same time on different host threads, each on its
 * own stream (aim_solve_batched). Their operator products become requests: requests of solves in
 * one size class (P = 64-128 or 256-512; larger grids keep their own launches) are fused into
 * one multi-context launch per grid-pass stage, as aim_matvec_multi does, on the batcher's own
 * stream, ordered against each solve's stream by CUDA events (no host thread waits for the GPU). A
 * request waits on the host until every solve of its class has submitted one, or max_wait_us. Each
 * solve's result is bit-identical to aim_solve of that context alone. aim_batcher_create makes a
 * batcher (its stream, events and launch buffers) on the current device; aim_batcher_destroy waits
 * for its work and frees it (no solve may be using it). aim_batcher_stats: products requested,
 * launches made, products that ran fused with others (host pointers, each may be NULL). */
typedef struct aim_batcher aim_batcher;
aim_status aim_batcher_create(int max_wait_us, aim_batcher** out);
void aim_batcher_destroy(aim_batcher* batcher);
aim_status aim_batcher_stats(aim_batcher* batcher, long long* products, long long* launches,
                             long long* fused_products);
/* aim_solve with its operator products going through `batcher` (see above); same arguments,
 * results and errors, plus AIM_ETIMEOUT when a fused launch's grid barrier gave up. One batched
 * solve per host thread at a time (AIM_ESTATE otherwise). */
aim_status aim_solve_batched(aim_batcher* batcher, aim_ctx* ctx, aim_op system, int nrhs,
                             const void* rhs, void* x, int x0_given, const aim_solve_opts* opts,
                             aim_solve_info* info, void* stream);

/* Device bytes that aim_setup followed by aim_reserve(nrhs, precision) would hold at their
 * peak, without touching the GPU (admission control; no counterpart in the paper). The count
 * runs the host part of the setup (grid, projections of Eq. 7 and the near-field pattern for
 * stencil->near_radius), so it is exact for the arrays, and takes every allocation in whole
 * 2 MiB allocator pages, so it is an upper bound on what the device commits. It does not
 * include a solve's Krylov basis (see aim_query_solve_bytes). Errors as for aim_setup's
 * argument checks (AIM_EINVAL). */
aim_status aim_query_bytes(const aim_geometry* geometry, const aim_grid* grid,
                           const aim_stencil* stencil, int nrhs, int precision, size_t* bytes);

/* Upper bound, like aim_query_bytes, on the device bytes a context holds after aim_setup and
 * aim_solve(nrhs, opts): the FP64 grid workspaces every solve reserves, the staging buffers, the
 * Krylov basis and reduction buffers for opts->restart, and the refinement vectors of a mixed
 * solve. Only opts->restart and opts->precision are read. */
aim_status aim_query_solve_bytes(const aim_geometry* geometry, const aim_grid* grid,
                                 const aim_stencil* stencil, int nrhs, const aim_solve_opts* opts,
                                 size_t* bytes);

/* One radix-16 pass of a batch of DFTs, on CUDA cores or on tensor cores (no counterpart in the
 * paper; for measurement). It answers whether the DFT stages of the grid product (Eq. 8 / Eq. 10)
 * should run on tensor cores: written as a dense contraction, the DFT-16 of one complex column is
 * the 32 x 32 real matrix [C S; -S C] (C = cos(2 pi k i/16), S = sin(2 pi k i/16)) times its 32
 * real and imaginary parts. Each CTA loads 4096 complex64 values of x, applies `passes` passes
 * to them in shared memory, and stores the result to y. A pass maps element i of column c (value
 * c + 256 i) to output k of column c (value 16 c + k):
 *     X_k(c) = sum_i x_i(c) t(c, i) exp(-2 pi j k i/16),  t(c, i) = exp(-2 pi j (c mod 16) i/256)/4.
 * variant: AIM_DFT_STAGE_CUDA_CORES (the product's register butterfly, FP32),
 *          AIM_DFT_STAGE_MMA_TF32 (mma.sync TF32, one product per term; the tensor core reads the
 *          top 19 bits of the FP32 data),
 *          AIM_DFT_STAGE_MMA_TF32X3 (mma.sync with the data split as hi = top 19 bits,
 *          lo = x - hi, and a_hi b_hi + a_hi b_lo + a_lo b_hi),
 *          AIM_DFT_STAGE_SPLIT_ONLY (the split variant's loads, twiddles, data split and stores
 *          without the products: each pass stores hi + lo = t(c, i) x_i(c) at value c + 256 i;
 *          its rate bounds any tensor-core pass fed from registers).
 * x, y: device pointers (current device), groups * 4096 interleaved complex64 values each,
 * 8-byte aligned; they may be the same buffer. groups in [1, 2^20], passes in [0, 2^20].
 * Returns AIM_EINVAL for a bad variant, size or pointer, before any launch. */
typedef enum {
  AIM_DFT_STAGE_CUDA_CORES = 0,
  AIM_DFT_STAGE_MMA_TF32 = 1,
  AIM_DFT_STAGE_MMA_TF32X3 = 2,
  AIM_DFT_STAGE_SPLIT_ONLY = 3
} aim_dft_stage_variant;

aim_status aim_dft_stage(int variant, int groups, int passes, const void* x, void* y, void* stream);

/* Launch accounting and kernel timing (no counterpart in the paper; for measurement).
 * aim_launch_count: kernels the library has enqueued in this process so far (all contexts).
 * aim_profile_start: from now on every launch is bracketed by two CUDA events recorded on
 * its own stream (adds two event records per launch).
 * aim_profile_stop: waits for the recorded events, writes per-kernel launch counts and
 * summed durations (ms) for up to max_stats kernels into `stats` (host array), sets *count,
 * and stops timing. `name` points to a static string. */
typedef struct {
  int kernel;
  const char* name;
  long long launches;
  double total_ms;
} aim_kernel_stat;

long long aim_launch_count(void);
aim_status aim_profile_start(void);
aim_status aim_profile_stop(aim_kernel_stat* stats, int max_stats, int* count);

const char* aim_status_str(aim_status status);

/* Reason for the most recent failure on the calling thread ("" if none). */
const char* aim_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* AIM_GB300_H */
