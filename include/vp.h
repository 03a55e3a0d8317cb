/*
 * vp.h -- C ABI of the GB300 voxel volume-potential library (libvp.so).
 *
 * The library evaluates, on one NVIDIA GB300 (sm_103a), the per-harmonic voxel
 * volume potential of the nested-mesh method for weakly nonlinear focused
 * ultrasound:
 *
 *     u = V_k[f],   u(x_i) = sum_{j != i} h^3 G_k(x_i - x_j) f(x_j) + S(k,h) f(x_i)
 *
 * with G_k(r) = exp(i k r) / (4 pi r) (Eq. 3.3), the midpoint rule off the diagonal
 * and the equal-volume-sphere integral S(k,h) = ((1 - i k a) e^{i k a} - 1) / k^2,
 * a = (3/(4 pi))^{1/3} h, on the diagonal (Eq. 3.9).  The sum is a 3-level Toeplitz
 * product evaluated by zero padding to a circulant of size M >= 2N - 1 per axis
 * and FFTs (Section 3.1).  Harmonic sources come from products of lower
 * harmonics (Eq. 2.6, written out in Eqs. 3.5-3.8); lower harmonics move between
 * nested grids by linear interpolation (Section 6).
 *
 * Conventions shared by every call
 * - Fields are complex64: interleaved (re, im) float32 pairs, C order (nx, ny, nz),
 *   z fastest, densely packed.  Field pointers are DEVICE pointers owned by the
 *   caller, 8-byte aligned.
 * - A grid is (n[3], origin[3], h): voxel (i,j,k) has centre origin + h*(i,j,k), in
 *   metres.
 * - Every call that takes a stream is asynchronous on that stream (a
 *   cudaStream_t passed as void*; NULL = the legacy default stream).  Host-side
 *   argument errors are detected before anything is enqueued.
 * - Every function returns an int status: VP_OK (0) or a negative VP_ERR_* code.
 *   Nothing throws across the ABI.  vp_status_string() names a code.
 * - Thread safety: distinct plans may be used from distinct host threads; one
 *   plan must not be used by two threads at once.
 *
 * Wavenumber and source coefficient (Section 2, readings of the paper):
 *   k_n = 2 pi n f0 / c0 + i alpha(n f0),
 *   alpha(f) [Np/m] = alpha0 [dB/m/MHz^eta] (f / 1 MHz)^eta / (20 log10 e),
 *   C_n = -beta omega^2 n^2 / (2 rho0 c0^4), omega = 2 pi f0
 *   (the minus sign of Eq. 3.2 is folded into C_n, so vp_apply is +int G f).
 */
#ifndef VP_H
#define VP_H

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define VP_API __attribute__((visibility("default")))
#else
#define VP_API
#endif

/* ---- status codes ------------------------------------------------------------ */
#define VP_OK               0
#define VP_ERR_ARG         -1  /* null pointer, non-positive size or spacing, bad harmonic */
#define VP_ERR_SIZE        -2  /* no FFT schedule for the requested embedding size        */
#define VP_ERR_NOMEM       -3  /* device allocation failed                                 */
#define VP_ERR_CUDA        -4  /* a CUDA runtime call or kernel launch failed              */
#define VP_ERR_NOT_NESTED  -5  /* restriction target not inside the source grid           */
#define VP_ERR_STATE       -6  /* call out of order (no staged source; spectrum not built) */
#define VP_ERR_TIMEOUT     -7  /* a bounded device wait expired (reported by vp_plan_check) */
#define VP_ERR_UNSUPPORTED -8  /* valid request outside what this build implements        */

typedef void* vp_stream_t; /* cudaStream_t */

typedef struct vp_grid {
    int n[3];          /* voxels per axis (x, y, z), each >= 1            */
    double origin[3];  /* centre of voxel (0,0,0), metres                  */
    double h;          /* voxel side, metres, > 0                          */
} vp_grid;

typedef struct vp_medium {
    double c0;      /* speed of sound, m/s                                   */
    double rho0;    /* density, kg/m^3                                       */
    double beta;    /* coefficient of nonlinearity                           */
    double alpha0;  /* attenuation prefactor, dB/m/MHz^eta (>= 0)            */
    double eta;     /* attenuation power-law exponent                        */
} vp_medium;

typedef struct vp_plan_s* vp_plan_t;

/* Optional plan overrides; zero-initialise and set only what you need. */
typedef struct vp_plan_opts {
    int m[3];           /* embedding size per axis; 0 = smallest even 5-smooth >= 2N     */
    int radix[3][8];    /* radix schedule per axis (product must equal M); 0-terminated,
                           all zero = default schedule                                    */
    int autotune;       /* nonzero and no m / radix given: time the default embedding
                           against the smallest even 5-smooth one, then (zform 0 and
                           M_z >= 512 on the two-level engine) every z-sweep form on the
                           winner (three applications each, on `stream`, with the
                           staging and layout asked for), and keep the fastest; cached
                           per grid shape, staging and layout                            */
    int zform;          /* form of the pipelined z sweep (two-level engine): VP_ZFORM_*;
                           0 = the form that keeps the most warps resident per SM.  A form
                           that is not compiled for M_z or does not fit in shared memory
                           is not used (the choice falls back as for 0)                  */
    int staging;        /* input staging of the 4-line z-sweep forms: 0 = one bulk
                           asynchronous copy per line and per spectrum octant line,
                           completion counted on an mbarrier, wherever every line starts
                           on a 16-byte boundary (even N_z), else as 1; 1 = 8-byte
                           cp.async per element (the other forms always stage this way) */
    int layout;         /* layout of the x forward sweep's output (the y forward sweep's
                           input): 0 = x rows grouped by 4 y-planes, element (x, y, z) at
                           ((y / 4) M_x + x) 4 N_z + (y % 4) N_z + z, where x and y both
                           run on the two-level engine and N_y is a multiple of 4, else
                           as 1; 1 = plain, (x N_y + y) N_z + z.  The grouped
                           layout keeps consecutive output rows of the x sweep 4 N_z
                           elements apart instead of N_y N_z, so that its writes stay
                           within a few pages (x forward on 600 x 600 x 640: 1.38
                           against 1.71 ms; the y forward reading it: 2.70 against
                           2.53 ms)                                                     */
    int test_expire_waits; /* test hook, 0 in normal use: nonzero makes the bulk-staged z
                           sweep issue none of its first copies, so that its bounded waits
                           expire (about one second each) and the next vp_plan_check
                           returns VP_ERR_TIMEOUT; the output of that apply is undefined */
} vp_plan_opts;

#define VP_ZFORM_AUTO   0
#define VP_ZFORM_TILE16 1  /* 16 lines a CTA (4 mirror groups), 256 threads              */
#define VP_ZFORM_TILE8  2  /* 8 lines a CTA (2 mirror groups), 256 threads, M_z >= 640   */
#define VP_ZFORM_TILE4  3  /* 4 lines a CTA (1 mirror group), 4 max(A, B) threads, M_z >= 512 */
#define VP_ZFORM_PAIR8  4  /* 8 lines, step 2 split over lane pairs, 512 threads, M_z = 1280 */
#define VP_ZFORM_TILE4T 5  /* 4 lines, the two steps' factors swapped (40 x 32, 32 x 24, 32 x 20),
                              M_z = 1280, 768, 640 */

typedef struct vp_plan_info {
    int n[3];
    int m[3];
    int radix[3][8];     /* 0-terminated                                                 */
    double k_re, k_im;   /* k_n                                                          */
    double c_n;          /* source coefficient C_n                                       */
    double self_re, self_im;      /* self-cell integral S(k_n, h)                        */
    unsigned long long workspace_bytes;  /* device bytes held by the plan               */
    int khat_ready;      /* 1 once vp_kernel_fft has been enqueued                       */
    int engine[3];       /* per axis: 1 two-level register FFT, 0 shared-memory radix passes */
    int zform;           /* z-sweep form asked for or chosen by the autotuner (VP_ZFORM_*) */
    int staging;         /* vp_plan_opts.staging of the plan                             */
    int group_y;         /* y-planes per group of the x sweep's output: 4 grouped, 1 plain */
} vp_plan_info;

/* ---- plans --------------------------------------------------------------------
 * vp_plan: create a plan for harmonic n (>= 1) on grid g (Section 6 algorithm, step 1:
 * one voxel mesh per harmonic).  Computes k_n and C_n, picks the embedding size M per
 * axis (Section 3.1 needs M >= 2N - 1, Section 6 uses 2N) and its FFT engine, and
 * allocates the plan's
 * device workspace (about 8 * (M_x N_y N_z + M_x M_y N_z) bytes) and the storage of
 * the kernel spectrum (8 * prod(M/2 + 1) bytes) on the current device.
 * Default M: the smallest length >= 2N - 1 compiled for the two-level register engine
 * (32, 64, 128, 192, 256, 320, 384, 512, 640, 768, 864, 1024, 1200, 1280) when it is at
 * most a third longer than the smallest even 2^a 3^b 5^c >= 2N, else that 5-smooth
 * length with the shared-memory radix-pass engine.  An explicit opts->radix schedule
 * selects the radix-pass engine for that axis.
 * `opts` may be NULL.  `stream` is used only when opts->autotune is set.
 * Errors: VP_ERR_ARG (null pointers, n[i] < 1, h <= 0, harmonic < 1, c0 <= 0,
 * rho0 <= 0, alpha0 < 0, f0 <= 0), VP_ERR_SIZE (M < 2N - 1, or an axis the FFT
 * engine cannot hold: M > 1536, or a radix schedule whose product is not M or that
 * uses a radix outside {2,3,4,5,8,16}), VP_ERR_NOMEM, VP_ERR_CUDA.
 * On error *out is set to NULL and nothing is leaked. */
VP_API int vp_plan(const vp_grid* g, int harmonic_n, double f0_hz, const vp_medium* m,
                   const vp_plan_opts* opts, vp_stream_t stream, vp_plan_t* out);

/* Release every device and host resource of the plan.  Synchronises the device
 * first (pending work that uses the plan completes).  NULL is accepted. */
VP_API int vp_destroy(vp_plan_t p);

/* Point an existing plan at another grid of the same voxel counts, harmonic, f0 and
 * medium (new spacing, origin, k_n, C_n and self cell), keeping its embedding size,
 * FFT schedule, tables and device workspace: a sequence of problems with equal N
 * (e.g. one instance after another at 6 voxels per wavelength) then needs no device
 * allocation.  The kernel spectrum becomes stale: call vp_kernel_fft before the next
 * vp_apply, and vp_source_assemble again.  Host-only; work already enqueued on the
 * plan keeps the state it was enqueued with only when it runs on the stream the next
 * vp_kernel_fft uses.  A batch created from the plan before the call refuses to run
 * afterwards (VP_ERR_STATE): create it again.  Errors: VP_ERR_ARG (as vp_plan), VP_ERR_UNSUPPORTED (harmonic
 * > 9), VP_ERR_SIZE (g->n differs from the plan's). */
VP_API int vp_plan_retarget(vp_plan_t p, const vp_grid* g, int harmonic_n, double f0_hz, const vp_medium* m);

/* Fill *info.  Errors: VP_ERR_ARG. */
VP_API int vp_plan_get_info(vp_plan_t p, vp_plan_info* info);

/* Device-side status of the plan's kernels.  The bulk-staged z sweep waits on its
 * copies with a bound of about one second (2^31 SM clock cycles) per wait; a CTA whose
 * wait expires records it in a device word of the plan, waits (again bounded) for its
 * copies still in flight and returns, leaving the context usable.  This call
 * synchronises `stream`, reads and clears that word, and returns VP_ERR_TIMEOUT if a
 * wait expired since the last check (the outputs of the applies in between are then
 * undefined), VP_ERR_STATE if a kernel refused a buffer that broke the alignment its
 * launcher checked, else VP_OK.  Errors: VP_ERR_ARG, VP_ERR_CUDA. */
VP_API int vp_plan_check(vp_plan_t p, vp_stream_t stream);

/* ---- kernel spectrum ----------------------------------------------------------
 * Build the spectrum of the circulant-embedded quadrature kernel (Section 6,
 * step 2b; Eq. 3.9): the lattice h^3 G_{k_n}(|d| h) for offsets d in (-N, N)^3 placed
 * at d mod M, the self-cell integral at d = 0 (FP64 on the device), zero at every
 * index no offset maps to; then its 3-D FFT.  The kernel is even in every axis, so
 * only the octant of frequencies [0, M/2]^3 is kept.  Phases k |d| h are formed in
 * FP64 and reduced modulo 2 pi before the single-precision sine/cosine.
 * Idempotent: later calls return VP_OK without work.  Uses a temporary device
 * buffer of 8 * M_x M_y M_z bytes, freed before return.
 * Errors: VP_ERR_ARG, VP_ERR_NOMEM, VP_ERR_CUDA. */
VP_API int vp_kernel_fft(vp_plan_t p, vp_stream_t stream);

/* Copy the octant spectrum (prod(M/2 + 1) complex64, C order) to/from a device
 * buffer, e.g. to cache it across processes.  Errors: VP_ERR_ARG, VP_ERR_STATE
 * (get before the spectrum was built), VP_ERR_CUDA. */
VP_API int vp_kernel_spectrum_get(vp_plan_t p, void* dst_device, vp_stream_t stream);
VP_API int vp_kernel_spectrum_set(vp_plan_t p, const void* src_device, vp_stream_t stream);

/* ---- source assembly -----------------------------------------------------------
 * f_n = C_n * sum_{m=1}^{n-1} p_m p_{n-m} (Eq. 2.6; Eqs. 3.5-3.8 for n = 2..5).
 * lower[m-1] is p_m on the plan's grid (device pointer, N voxels), n_lower must be
 * n - 1 (>= 1).
 * flags & VP_SRC_CONJ: the full cascade of Eq. 2.5 instead, which keeps the products
 *   with harmonics above n:  f_n = C_n [ sum_{m=1}^{n-1} p_m p_{n-m}
 *   + 2 sum_{m=n+1}^{N_h} p_m conj(p_{m-n}) ];  lower[m-1] = p_m for m = 1..N_h with
 *   n_lower = N_h (n <= N_h <= 8, N_h >= 2), every entry non-NULL (p_n itself enters
 *   through p_{2n} conj(p_n) when 2n <= N_h); any harmonic n >= 1.  The source is
 *   formed in its own pass (not fused into the first sweep).
 * f_out != NULL: write f_n (N voxels, complex64) there.
 * f_out == NULL: fuse the assembly with the zero padding and the first FFT sweep of
 *   vp_apply, leaving the transformed source in the plan's workspace; the next
 *   vp_apply(p, NULL, u, ...) on the same stream consumes it.
 * Errors: VP_ERR_ARG (null plan or field pointer, n_lower out of range, unknown flags),
 * VP_ERR_CUDA. */
#define VP_SRC_CONJ 1
VP_API int vp_source_assemble(vp_plan_t p, const void* const* lower, int n_lower, int flags,
                              void* f_out, vp_stream_t stream);

/* ---- source assembly from lower harmonics on their own nested grids -----------------
 * The source f_n of vp_source_assemble (Eq. 2.6) when p_m lives on a grid of its own
 * (Section 6, steps 2a-2b): lower[m-1] is p_m on grids[m-1] (device pointer,
 * grids[m-1].n voxels), for m = 1..n-1, n_lower = n - 1.  One kernel restricts every p_m
 * to the plan's grid (the interpolation of vp_restrict_to_nested_box: linear, or
 * quadratic with flags & VP_RESTRICT_QUADRATIC) and forms f_n from the restricted values
 * there; the restricted fields are never stored.  Same result as
 * vp_restrict_to_nested_box of each p_m followed by vp_source_assemble (up to the order
 * of the FP32 sums).  Every plan voxel centre must lie within each source box, as for
 * vp_restrict_to_nested_box without VP_RESTRICT_ZERO_OUTSIDE.
 * f_out != NULL: write f_n (N voxels, complex64) there.
 * f_out == NULL: stage f_n for the next vp_apply(p, NULL, u, ...) on the same stream
 *   (its first FFT sweep runs here, from the plan's workspace).
 * Errors: VP_ERR_ARG (null plan, array or field pointer, n_lower != n - 1, n < 2, a bad
 * grid, unknown flags), VP_ERR_NOT_NESTED, VP_ERR_UNSUPPORTED (plan grid with more than
 * 65535 voxels along x or y), VP_ERR_CUDA. */
VP_API int vp_source_from_nested(vp_plan_t p, const vp_grid* grids, const void* const* lower, int n_lower,
                                 int flags, void* f_out, vp_stream_t stream);

/* ---- volume potential ----------------------------------------------------------
 * u = V_{k_n}[f] (Eq. 3.9 via the circulant embedding of Section 3.1): zero pad f to
 * M, forward 3-D FFT, multiply by the kernel spectrum, inverse FFT, crop to N.
 * f == NULL uses the source staged by vp_source_assemble(..., f_out = NULL).
 * u must not alias f.  Errors: VP_ERR_ARG (null plan or u), VP_ERR_STATE (spectrum
 * not built, or f == NULL with nothing staged), VP_ERR_CUDA. */
VP_API int vp_apply(vp_plan_t p, const void* f, void* u, vp_stream_t stream);

/* ---- restriction between nested grids ------------------------------------------
 * dst_field = linear (trilinear) interpolation of src_field, given on grid src, at
 * the voxel centres of grid dst (Section 6, step 2a).  For a target coordinate on
 * one axis, t = (x - o_src)/h_src, i0 = floor(t) clamped to [0, N-2], w = t - i0;
 * the result is the tensor product of (1-w) v[i0] + w v[i0+1].  Axis positions are
 * held as exact 40-bit fixed-point numbers, T_i = round(a 2^40) + i round(b 2^40) with
 * a = (o_dst - o_src)/h_src and b = h_dst/h_src formed in FP64 (round half away from
 * zero), and every index decision is taken on T_i; weights are applied in FP32.
 * Every target centre must lie within the box spanned by the source centres (a
 * relative slack of 1e-9 voxel is allowed); otherwise VP_ERR_NOT_NESTED unless
 * flags & VP_RESTRICT_ZERO_OUTSIDE, which writes zero there instead.
 * flags & VP_RESTRICT_QUADRATIC selects quadratic interpolation instead (the higher-
 * order inter-mesh interpolation Section 6 leaves as an option): per axis the Lagrange
 * quadratic through the three nearest source centres, c = floor(t + 1/2) clamped to
 * [1, N-2], u = t - c, weights (u(u-1)/2, 1-u^2, u(u+1)/2) on v[c-1], v[c], v[c+1];
 * an axis of two voxels stays linear.  Exact for fields quadratic along each axis.
 * Errors: VP_ERR_ARG, VP_ERR_NOT_NESTED, VP_ERR_CUDA. */
#define VP_RESTRICT_ZERO_OUTSIDE 1
#define VP_RESTRICT_QUADRATIC 2
VP_API int vp_restrict_to_nested_box(const vp_grid* src, const void* src_field, const vp_grid* dst,
                                     void* dst_field, int flags, vp_stream_t stream);

/* ---- field vector operations ----------------------------------------------------------
 * Complex64 device arrays of n elements; FP32 arithmetic, FP64 accumulation for dot.
 * Used by the fixed-point iteration of the full cascade and the VIE solver.
 * vp_vec_axpby: out = a x + b y (y may be NULL: out = a x); out may alias x or y.
 * vp_vec_mul:   out = x * y elementwise; out may alias x or y.
 * vp_vec_dot:   out[0] + i out[1] = sum_i (conj_x ? conj(x_i) : x_i) y_i, to host
 *               memory (synchronises the stream).
 * Errors: VP_ERR_ARG (n < 1, null pointers), VP_ERR_CUDA. */
VP_API int vp_vec_axpby(long long n, double a_re, double a_im, const void* x, double b_re, double b_im,
                        const void* y, void* out, vp_stream_t stream);
VP_API int vp_vec_mul(long long n, const void* x, const void* y, void* out, vp_stream_t stream);
VP_API int vp_vec_dot(long long n, const void* x, const void* y, int conj_x, double out[2], vp_stream_t stream);

/* ---- inhomogeneous medium: volume integral equation (Section 7) -----------------------
 * Solves  p(x) - int G_{k_n}(x - y) q(y) p(y) dy = b(x)  (Eqs. 7.1-7.5 with the contrast
 * q(y) = k_n(y)^2 - kbar_n^2, zero where the medium is the background of the plan), in
 * the quadrature of vp_apply: (I - V_{k_n} Q) p = b on the plan's grid.  For n = 1, b is
 * the incident field; for n >= 2 it is the potential of the harmonic's source.
 * BiCGStab, two operator applications per iteration (each: q x, vp_apply, x - V[q x]),
 * inner products in FP64.  q, b: device complex64 (N voxels); x: in the initial guess,
 * out the solution.  Stops when ||b - A x|| <= tol ||b|| (*relres, host) or after
 * max_iter iterations (*iters, host; either may be NULL); a breakdown of the recurrence
 * returns the current iterate with its residual.  Allocates 8 N-voxel fields from the
 * stream-ordered pool and synchronises the stream once per inner product.
 * Errors: VP_ERR_ARG (null pointers, tol <= 0, max_iter < 1), VP_ERR_STATE (spectrum not
 * built), VP_ERR_NOMEM, VP_ERR_CUDA. */
VP_API int vp_vie_solve(vp_plan_t plan, const void* q, const void* b, void* x, double tol, int max_iter,
                        int* iters, double* relres, vp_stream_t stream);

/* ---- integration-domain selection (Section 5) -------------------------------------
 * Smallest voxel box D of the N^3 field f (complex64, device) outside which
 * Q(x) = log10(|f(x)| / max|f|) < q0 (Section 5's domain-convergence study; q0 <= 0):
 * box[0..2] = first and box[3..5] = last index per axis, inclusive, written to host
 * memory.  Squares |f|^2 are formed in FP64 from the FP32 parts and compared with
 * 10^(2 q0) max|f|^2 (so a field that is zero everywhere gives the whole grid).  If
 * max_abs is not NULL it receives max|f|.  Synchronises `stream`.
 * Errors: VP_ERR_ARG (null pointers, n[i] < 1, q0 > 0 or not finite), VP_ERR_CUDA. */
VP_API int vp_q0_box(const int n[3], const void* f, double q0, int box[6], double* max_abs, vp_stream_t stream);

/* ---- incident field (input generator) -------------------------------------------
 * p1 on grid g from a bowl of focal length l and aperture radius R driven at f0 with
 * surface pressure p0, as a monopole sum over n_points bowl points (Eq. 3.10):
 *   p1(x) = -2 i k_1 p0 (A / n_p) sum_i G_{k_1}(x - r_i),  A = 2 pi l (l - sqrt(l^2 - R^2)).
 * (Reading: uniform normal velocity p0/(rho0 c0) in the Rayleigh integral; the paper
 * normalises to a radiated power instead.)  points: DEVICE pointer to n_points x 3
 * float64 (x, y, z).  Distances and phases in FP64, reduced modulo 2 pi before the
 * single-precision sine/cosine; accumulation in FP32 per point block, FP64 across
 * blocks.  Errors: VP_ERR_ARG, VP_ERR_CUDA. */
VP_API int vp_incident_field(const vp_grid* g, const double* points, int n_points, double l,
                             double R, double f0_hz, double p0, const vp_medium* m, void* out,
                             vp_stream_t stream);

/* ---- batched evaluation -------------------------------------------------------------
 * Many independent evaluations (e.g. many transducer configurations, each with its own
 * nested grids) bound once and run together.  Item i computes u[i] = V_{k_n}[f_i] with
 * plans[i]: f_i = f[i] when f != NULL and f[i] != NULL, otherwise the source of Eq. 2.6
 * assembled from lower[i * 8 + 0 .. i * 8 + n - 2] (p_1 .. p_{n-1} on the plan's grid;
 * rows of 8 pointers).  Items whose plans share the embedding size on every axis, run
 * the two-level engine on every axis and agree on f vs source form one group; each
 * group runs as one launch per FFT sweep over all its items (each CTA finds its item
 * in a per-sweep offset table), so a batch of uneven grids needs a handful of
 * launches instead of five per item.  In a group whose items each give the z sweep
 * at least 8 tiles of 16 lines per SM, that sweep runs item by item with the
 * single-plan kernel (the column sweeps stay grouped).  Other items run one plan at a
 * time.  All
 * pointers are device pointers bound at creation; vp_batch_run recomputes from their
 * current contents, so a stream capture of vp_batch_run replays correctly.  A plan may
 * appear at most once per batch (items share nothing but read-only inputs); kernel
 * spectra must be built (vp_kernel_fft) before vp_batch_run.
 * Errors: VP_ERR_ARG (count < 1, null plan or output, a plan listed twice, a missing
 * source field), VP_ERR_STATE (spectrum not built), VP_ERR_NOMEM, VP_ERR_CUDA. */
typedef struct vp_batch_s* vp_batch_t;
VP_API int vp_batch_create(int count, const vp_plan_t* plans, const void* const* f, const void* const* lower,
                           void* const* u, vp_batch_t* out);
/* The same as vp_batch_create with the plans first, as the batched call of the interface
 * sketch names it (plans, count, ...); identical behaviour and errors. */
VP_API int vp_batch_plan(const vp_plan_t* plans, int count, const void* const* f, const void* const* lower,
                         void* const* u, vp_batch_t* out);
VP_API int vp_batch_run(vp_batch_t b, vp_stream_t stream);
VP_API int vp_batch_destroy(vp_batch_t b);

/* ---- allocation-free volume potential --------------------------------------------
 * The paper has no counterpart to this entry point; it exists for callers that cannot
 * call cudaMalloc: code running while a stream is captured into a CUDA graph
 * (cudaMalloc/cudaFree are not capturable, and cudaFree synchronises the device),
 * applications whose device memory is owned by another allocator that already holds
 * it, and latency-bound loops that cannot afford the device-wide synchronisation of
 * cudaMalloc/cudaFree.
 *
 * vp_apply_static computes the same u = V_{k_n}[f] as vp_plan + vp_kernel_fft + vp_apply,
 * for grids of at most VP_STATIC_MAX_N voxels per axis, on the smallest even 5-smooth
 * embedding M >= 2N with the radix-pass FFT engine (vp_plan may pick another embedding
 * and engine), so the two agree to FP32 rounding, not bit for bit.  Every intermediate
 * lives in one fixed-size __device__ array inside libvp.so (about 18.2 MiB, held by
 * every GPU that loads the library until the process exits).  It calls no cudaMalloc,
 * cudaFree or other allocating routine.  The caller passes f and u (device pointers,
 * complex64, N voxels each, not aliased); the kernel spectrum is rebuilt on every call.
 * - The first call in a CUDA context looks up the array's device address
 *   (cudaGetSymbolAddress) with the device current, and caches it for that device and
 *   context; make that first call before any stream capture (again after a
 *   cudaDeviceReset, which gives the device a new context).
 * - Every call on a device shares the array and rewrites everything it later reads,
 *   so no state carries over between calls; calls whose GPU work overlaps (other
 *   streams, other host threads) race on the array and must be serialised.
 * Errors: VP_ERR_ARG (null pointers, n[i] < 1, h <= 0, harmonic < 1, f0 <= 0, c0 <= 0,
 * rho0 <= 0, alpha0 < 0, or a non-finite h, f0, c0, rho0, alpha0, beta or eta),
 * VP_ERR_SIZE (an axis longer than VP_STATIC_MAX_N), VP_ERR_CUDA. */
#define VP_STATIC_MAX_N 64
VP_API int vp_apply_static(const vp_grid* g, int harmonic_n, double f0_hz, const vp_medium* m,
                           const void* f, void* u, vp_stream_t stream);

/* ---- diagnostics ----------------------------------------------------------------- */
/* Static, NUL-terminated name of a status code. */
VP_API const char* vp_status_string(int status);

/* Per-kernel timing of vp_apply / vp_source_assemble: when enabled, the plan records
 * a CUDA event pair around each FFT sweep it launches, on the launching stream.
 * vp_profile_read returns, for sweep s in 0..4 (x forward with source, y forward,
 * z forward + spectrum multiply + z inverse, y inverse, x inverse), the summed
 * milliseconds and launch counts since the last reset, synchronising on the
 * recorded events.  Errors: VP_ERR_ARG, VP_ERR_CUDA. */
VP_API int vp_profile_enable(vp_plan_t p, int on);
VP_API int vp_profile_read(vp_plan_t p, double ms[5], int count[5], int reset);

/* Library build identification string (static): "libvp <version> sm_103a src <digest>",
 * where <digest> is the SHA-256 prefix of the sources the library was built from. */
VP_API const char* vp_version(void);

#ifdef __cplusplus
}
#endif
#endif /* VP_H */
