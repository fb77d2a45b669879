/*
 * p3m.h -- C ABI of the GB300 (sm_103a) P3M space-charge library.
 *
 * The library evaluates the particle-particle-particle-mesh (P3M) space-charge force of
 * Wyssling & Adelmann, "On Boundary Conditions in the sub-mesh interaction of the
 * Particle-Particle-Particle-Mesh Algorithm" (arXiv 2103.02046), and pushes particles with
 * the variational leapfrog of the same paper:
 *
 *   F_i = F^S_i + F^L_i                                   (eq. (eom_p3m_coord), right-hand side)
 *   F^S_i = sum_{j != i, |xi_i - xi_j| < r_c} k_e q^2 [erfc(a r)/r + (2a/sqrt(pi)) e^{-a^2 r^2}]
 *           (xi_i - xi_j)/r^2                             (eq. (summation_short), G^S of eq. (ewald_split))
 *   F^L_i = -q sum_g phi_g grad_xi W(x_g - xi_i)          (eq. (eom_p3m_coord), first term)
 *   phi_g = k_e sum_g' Q_g' [G^L(x_g - x_g') - G^L(x_g - S(x_g'))]
 *                                                         (eq. (phi_L) with eq. (GreenFunc_planar_cathode))
 *   Q_g   = q sum_i W(x_g - xi_i)                         (eq. (rho_L))
 *
 * with G^L(r) = erf(a r)/r, W the TSC (or cloud-in-cell) assignment function, S the mirror
 * map at the cathode plane z = z_cathode, and k_e = 1/(4 pi eps0).
 *
 * Conventions for every entry point:
 *   * Units are SI. Particle arrays are caller-owned, contiguous, row-major [n][3] float64
 *     in DEVICE memory (positions x in m, momenta p in kg m/s, forces in N).
 *   * The context owns all scratch memory. Only p3m_create allocates (mesh, spectra, sort
 *     buffers, FFT plans, adjoint checkpoints). No other call allocates or frees.
 *   * Every call is asynchronous and stream-ordered on the context's stream. Host-detectable
 *     errors (null pointers, bad parameters, n > n_max) are returned at once. Errors found on
 *     the device (a particle outside the mesh's valid range or below the cathode, a NaN
 *     position, a bounded wait that ran out) are latched in a device-visible word and
 *     returned by the next call or by p3m_sync. Nothing traps or aborts; after an error the
 *     context stays usable.
 *   * Status codes are p3m_status; p3m_last_error gives a message for the last failure.
 */
#ifndef P3M_H
#define P3M_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  P3M_OK = 0,
  P3M_EINVAL = 1,   /* bad argument or parameter */
  P3M_ENOMEM = 2,   /* device allocation failed in p3m_create */
  P3M_ECUDA = 3,    /* a CUDA runtime call failed */
  P3M_ECUFFT = 4,   /* a cuFFT call failed */
  P3M_ERANGE = 5,   /* a particle lies outside the mesh's valid range or below the cathode */
  P3M_ETIMEOUT = 6, /* a bounded device-side wait ran out */
  P3M_ESTATE = 7    /* call not valid in the context's current state */
} p3m_status;

typedef enum { P3M_FP64 = 0, P3M_FP32_MIXED = 1 } p3m_precision;

/* Problem statement (Sec. 2.4: macro-particles, mesh; Sec. 2.2: split; Sec. 3.1: cathode). */
typedef struct p3m_params {
  int32_t n[3];          /* mesh nodes per axis, x, y, z (each in [8, 1024]) */
  double lo[3];          /* position of node 0 [m]; node g sits at lo + g*h (Sec. 2.4.2) */
  double h[3];           /* mesh spacing per axis [m] */
  double rc_over_h;      /* short-range cutoff r_c = rc_over_h * max_d h_d; >= 0.25 */
  double kappa;          /* Ewald parameter a = kappa / r_c (eq. (ewald_split)) unless alpha > 0 */
  double alpha;          /* explicit Ewald parameter [1/m]; <= 0 selects kappa / r_c */
  int32_t assign_order;  /* 1 = cloud-in-cell (eq. (interpolation_splines_b0)), 2 = TSC */
  int32_t pm_bc;         /* 0 = open boundaries, 1 = grounded cathode plane z = z_cathode in the
                            long-range solve, 2 = grounded box: phi = 0 on the mesh's six faces
                            (nodes 0 and n_d - 1), discrete-Laplacian long range of eq. (def_G_L);
                            FP64 path, pp_bc = 0, influence = 0; every particle's assignment
                            support must stay on interior nodes (else P3M_ERANGE) */
  int32_t pp_bc;         /* 0 = short range in free space (the paper's prescription),
                            1 = cathode images also in the short-range sum */
  double z_cathode;      /* cathode plane z [m] (eq. (symmetry_planar_cathode) at z = z_cathode) */
  int32_t influence;     /* 0 = sampled G^L; optimal influence function of eq. (Ghfinal) as a
                            factor on the sampled kernels: 1 = principal alias only (1/U^2),
                            2 = alias sums over |m_d| <= 2 (computed once in p3m_create) */
  int32_t precision;     /* p3m_precision. P3M_FP64: positions, separations, pair decisions
                            (r^2 < r_c^2), sums, mesh and x-y transforms in FP64; the short-range
                            pair function erfc/exp in double-float arithmetic (pairs of FP32
                            numbers, relative error about 5e-14 at kappa = 3) for kappa <= 6.5,
                            FP64 above; the z transforms and the Green's-function multiply in
                            double-float (non-deterministic contexts, Mz a power of two in
                            [64, 2048]), else FP64; forces match an FP64 evaluation to 1e-12. P3M_FP32_MIXED: FP32 short
                            range with exact FP32 separations and compensated sums, FP32 mesh and
                            transforms, FP64 positions, results and reductions; forces match the
                            FP64 path to about 2e-7 (bounded by 1e-5) */
  int32_t deterministic; /* 1 = run-to-run identical results (FP64 path, pm_bc 0 or 1): particles
                            in a fixed order within each cell, every ordered pair evaluated by
                            its own particle without reductions, node charges summed exactly in
                            128-bit fixed point, energies and emittances in fixed-order
                            reductions. 0 = the faster unordered reductions (default) */
  int32_t adj_slots;     /* checkpoint slots for p3m_backward (0 disables the reverse pass) */
  int32_t adj_segment;   /* steps per checkpoint segment in p3m_backward */
  double q;              /* macro-particle charge [C] (all particles equal) */
  double mass;           /* macro-particle mass [kg] */
  int32_t force_diff;    /* long-range force: 0 = analytic derivative of the assignment function
                            (the variational force of eq. (eom_p3m_coord), default), 1 = central
                            differences of the mesh potential, -(phi_{g+e} - phi_{g-e}) / 2h,
                            interpolated with the assignment function (conserves momentum; not
                            variational, so p3m_force_vjp and p3m_backward refuse it with
                            P3M_ESTATE); every particle's assignment support must then keep one
                            node off the mesh edge (else P3M_ERANGE) */
  int32_t search_rows;   /* short-range search cells (Sec. 2.4, the cell list that finds the pairs
                            of eq. (summation_short)): rows per cutoff length in y and z, 1, 2 or
                            3; 0 (default) chooses from the mesh and n_max: 3 when the estimated
                            neighbour count (n_max particles over the mesh volume, per cutoff
                            sphere) is 200 or more, else 2, or 1 where the cell budget
                            (max(4 n_max, 2^20) cells) leaves no room for rows r_c/2 wide with
                            x cells r_c/4. Results do not depend on it beyond rounding order */
  int32_t search_xcells; /* x cells per cutoff length, 1, 2, 4, 8, 16 or 32; 0 (default) chooses
                            (4, or 16 with 3 rows, fewer where the cell budget requires). A
                            layout with an explicit search_rows or search_xcells over the cell
                            budget gives P3M_EINVAL */
} p3m_params;

typedef struct p3m_ctx p3m_ctx; /* opaque; owns all scratch memory */

/* Fills defaults: n = 64^3, TSC, rc_over_h = 2, kappa = 3, open boundaries, FP64,
 * q = 1e-15 C, mass = (q/e) m_e, adj_slots = adj_segment = 0. Returns P3M_EINVAL on NULL. */
p3m_status p3m_default_params(p3m_params* p);

/* Mesh over the particles' bounding box (a reading: the paper leaves the mesh extent open):
 * per axis, with [a_d, b_d] the bounding box of x (device [n][3] float64),
 * h_d = (b_d - a_d)/(n_d - 5) and lo_d = a_d - 2 h_d, so every particle keeps two nodes of
 * margin for TSC. Reads inout->n, writes inout->lo and inout->h. Synchronous on `stream`
 * (a cudaStream_t, may be NULL for the legacy default stream); needs no context and uses a
 * 64-byte device buffer that it allocates and frees itself. EINVAL if n < 1, any n_d < 8,
 * or the box is degenerate or not finite. */
p3m_status p3m_auto_mesh(const double* x, int64_t n, p3m_params* inout, void* stream);

/* Validates params, allocates every buffer for up to n_max particles, creates the FFT
 * plans and builds the Green's-function spectra (eq. (phi_L), eq. (GreenFunc_planar_cathode)).
 * `stream` (cudaStream_t, may be NULL) becomes the context's stream. *out is set on success.
 * EINVAL: bad params or n_max outside [1, 2^31 - 1]; ENOMEM / ECUFFT / ECUDA on failure
 * (nothing is leaked). */
p3m_status p3m_create(const p3m_params* params, int64_t n_max, void* stream, p3m_ctx** out);

/* Releases every resource of ctx (waits for its stream first). NULL is accepted. */
p3m_status p3m_destroy(p3m_ctx* ctx);

/* Sets the stream later calls are ordered on (cudaStream_t, may be NULL). */
p3m_status p3m_set_stream(p3m_ctx* ctx, void* stream);

/* Charge assignment, eq. (rho_L): node charges Q_g = q sum_i W(x_g - xi_i) for the n
 * positions x (device [n][3] float64), kept in ctx. Bins and sorts the particles first. */
p3m_status p3m_deposit(p3m_ctx* ctx, const double* x, int64_t n);

/* Long-range mesh potential from the last deposit, eq. (phi_L): phi = k_e (K_f * Q - K_i * Q_rev)
 * by doubled-mesh FFT convolution (K_i only with pm_bc = 1). ESTATE if nothing was deposited. */
p3m_status p3m_solve(p3m_ctx* ctx);

/* Copies a mesh quantity to caller device memory `out` (float64, n_z*n_y*n_x, x fastest):
 * which = 0 node charges Q [C], which = 1 mesh potential phi [V]; which = 2, 3, 4 (FP32 path,
 * after a p3m_forces call that included the long range) the forward differences of the mesh
 * potential along x, y, z, D_d phi(g) = phi(g + e_d) - phi(g) [V], which the FP32 path convolves
 * directly (difference kernels, eq. (phi_L)) and interpolates with the assignment function
 * (eq. (eom_p3m_coord) by summation by parts); at g_d = n_d - 1 phi(g + e_d) is the open-boundary
 * potential one node outside the mesh. ESTATE if not computed. */
p3m_status p3m_get_mesh(p3m_ctx* ctx, int32_t which, double* out);

/* One P3M force evaluation, eq. (eom_p3m_coord) right-hand side: f = F^S + F^L for the n
 * positions x (device [n][3] float64), written to f (device [n][3] float64, caller-owned,
 * may not alias x). energy (nullable, device float64[2]) receives the short-range energy
 * (1/2) q sum_i phi^S_i and the long-range mesh energy (1/2) sum_g Q_g phi_g [J].
 * parts selects the terms: 1 = short range only, 2 = long range only, 3 = both.
 * Invalid particles get f = 0 and latch ERANGE. */
p3m_status p3m_forces_ex(p3m_ctx* ctx, const double* x, int64_t n, double* f, double* energy,
                         int32_t parts);
p3m_status p3m_forces(p3m_ctx* ctx, const double* x, int64_t n, double* f, double* energy);

/* In-cutoff ordered pair count (and short-range image pairs) of the last force evaluation
 * that included the short range. Synchronises the context's stream. */
p3m_status p3m_pair_count(p3m_ctx* ctx, int64_t* pairs, int64_t* image_pairs);

/* Candidate tests of the short range on the particles of the last binning (the last forces,
 * deposit or push call): the number of (particle, record) pairs the neighbour search hands to
 * the distance test. Each unordered pair is looked at from one side only, so this bounds
 * pairs / 2 from above; the ratio is the search's efficiency. The FP32 path recounts them from
 * the sorted records on request (its short range carries no counter); the FP64 path's short
 * range counts as it runs (so there: the last evaluation that included the short range).
 * *candidates is written on success; synchronises the context's stream. P3M_EINVAL for a NULL
 * argument. */
p3m_status p3m_candidate_count(p3m_ctx* ctx, int64_t* candidates);

/* The short-range search layout the context uses (Sec. 2.4, the cell list behind
 * eq. (summation_short)): cell rows per cutoff length in y and z (1, 2 or 3) and x cells per
 * cutoff length, as chosen at p3m_create from search_rows / search_xcells. Host only, no device
 * work. P3M_EINVAL for a NULL argument. */
p3m_status p3m_search_layout(const p3m_ctx* ctx, int32_t* rows, int32_t* xcells);

/* Leapfrog, eq. (leapfrog) with the Stoermer form of eq. (eom_p3m_coord), as kick-drift-kick
 * (a reading: the paper leaves the start-up open):
 *   p += dt/2 F(x);  x += dt p / mass;  p += dt/2 F(x)   per step, nsteps >= 0 steps.
 * x, p: device [n][3] float64, updated in place. f (nullable, device [n][3] float64): if given,
 * it holds F(x0) on entry (reused, not recomputed) and F(x_end) on exit; if NULL, F(x0) is
 * computed and the forces stay in the context's scratch. */
p3m_status p3m_push(p3m_ctx* ctx, double* x, double* p, int64_t n, double dt, int32_t nsteps,
                    double* f);

/* p3m_push with the entry force made optional: f (device [n][3] float64, required) holds F(x0)
 * on entry if f_valid != 0, else F(x0) is computed into it; on exit it holds F(x_end). */
p3m_status p3m_push_ex(p3m_ctx* ctx, double* x, double* p, int64_t n, double dt, int32_t nsteps,
                       double* f, int32_t f_valid);

/* Vector-Jacobian product of the force map: out = (dF/dx)^T w for positions x and cotangent
 * w (all device [n][3] float64). The long-range part uses the symmetry of the solve
 * (both Green's functions are symmetric in their arguments), so it costs one extra solve. */
p3m_status p3m_force_vjp(p3m_ctx* ctx, const double* x, int64_t n, const double* w, double* out);

/* Reverse pass of p3m_push: given dJ/dx_T (gx_T) and dJ/dp_T (gp_T) for the state after
 * nsteps steps from (x0, p0), writes dJ/dx_0 (gx0) and dJ/dp_0 (gp0). States are
 * re-computed from checkpoints taken every ckpt_every steps (0 = adj_segment; at most
 * adj_segment, the length of the segment buffer p3m_create sizes; needs
 * adj_slots * ckpt_every >= nsteps). All arrays device [n][3] float64. ESTATE if the
 * context was created with adj_slots = 0; EINVAL if ckpt_every is outside [0, adj_segment] or
 * nsteps exceeds the checkpoint budget. */
p3m_status p3m_backward(p3m_ctx* ctx, const double* x0, const double* p0, int64_t n, double dt,
                        int32_t nsteps, int32_t ckpt_every, const double* gx_T,
                        const double* gp_T, double* gx0, double* gp0);

/* Normalised rms emittance eps_u = sqrt(<du^2><dp_u^2> - <du dp_u>^2)/(mass c), u = x, y, z
 * (a reading: the paper names emittance but does not define it). eps3: device float64[3].
 * gx, gp (nullable, device [n][3]): gradient of eps_x + eps_y + eps_z. */
p3m_status p3m_emittance(p3m_ctx* ctx, const double* x, const double* p, int64_t n, double* eps3,
                         double* gx, double* gp);

/* Largest n accepted by p3m_emittance_noalloc. */
#define P3M_NOALLOC_MAX_N 16777216

/* The same normalised rms emittance (and optional gradient) as p3m_emittance, for callers that
 * cannot allocate device memory: code that runs inside a host application owning every byte of
 * the device through its own allocator or a fixed memory budget, monitoring hooks called from a
 * simulation loop where an allocation could stall or fail mid-run, and code that must not touch
 * the CUDA allocator at all. The paper has no counterpart; this is a library service.
 *   x, p: device [n][3] float64 (caller-owned); mass [kg] > 0; eps3: device float64[3];
 *   gx, gp: nullable device [n][3] float64 for the gradient of eps_x + eps_y + eps_z;
 *   stream: cudaStream_t (may be NULL).
 * It needs no context and allocates nothing: its scratch is a fixed 512 KiB array in device
 * memory that every GPU loading the library holds until the process exits. Its first call in a
 * CUDA context (normally a device's primary context, with that device current) looks up the
 * array's address and keeps it for that context; make that first call before any stream capture. Every call shares the array; each call writes every
 * slot it later reads, so no state carries over, but calls that overlap on the GPU (other
 * streams, no ordering between them) race and must not be issued. The sums are combined in a
 * fixed order, so results are reproducible run to run.
 * Errors: EINVAL for NULL x/p/eps3, n < 2, mass <= 0 or n > P3M_NOALLOC_MAX_N; ECUDA if the
 * scratch address cannot be obtained or one of this call's launches fails (an error left
 * pending by the caller's earlier work is neither reported nor cleared). Asynchronous on
 * `stream`. */
p3m_status p3m_emittance_noalloc(const double* x, const double* p, int64_t n, double mass,
                                 double* eps3, double* gx, double* gp, void* stream);

/* Measurement utility (no counterpart in the paper): launches an FP32 fused-multiply-add chain
 * kernel on the current device (8 blocks of 256 threads per SM, 8 independent chains of `iters`
 * steps per thread; packed != 0 uses the two-wide FP32 instructions) on `stream` and writes the
 * launch's flop count (FMA = 2 flops) to *flops (host). Time the launch with events on the same
 * stream to measure the FP32 pipe's throughput, the denominator of the short range's roofline.
 * Allocates nothing. EINVAL for NULL flops or iters < 1; ECUDA if the launch fails. */
p3m_status p3m_fp32_probe(int32_t packed, int32_t iters, double* flops, void* stream);

/* Waits for the context's stream and returns any latched device error (then clears it). */
p3m_status p3m_sync(p3m_ctx* ctx);

/* Stage times of the last force evaluation in ms (CUDA events; synchronises):
 * [0] bin+sort, [1] short range, [2] deposit, [3] solve, [4] interpolation+combine, [5] total. */
p3m_status p3m_get_timings(p3m_ctx* ctx, double* ms, int32_t cap, int32_t* count);

/* Message for the last failure on ctx (never NULL; valid until the next call on ctx). */
const char* p3m_last_error(const p3m_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* P3M_H */
