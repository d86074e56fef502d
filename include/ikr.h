/*
 * ikr.h - C ABI of the GB300 (sm_103a) inexact-Krylov linear-response library.
 *
 * The library solves the Dyson equation of density-functional perturbation
 * theory,  E drho = b  with  E = 1 - chi0 K  (the dielectric adjoint,
 * Sec. 2.2 and eq. dyson_discretised), by the inexact GMRES of Algorithm 1
 * whose inner Sternheimer equations (eq. discretised_sternheimer) are solved
 * by CG to adaptively chosen tolerances (Theorem inexact_gmres_dyson, Table
 * strategies, Table strategies_k).  Every step runs in the library's own CUDA
 * kernels on one GPU; the host only runs the GMRES bookkeeping (Givens
 * rotations, the smallest singular value of the (i+1) x i Hessenberg matrix)
 * and the tolerance rule.
 *
 * Conventions shared by all calls
 *  - Cell: lattice[3*i + j] is Cartesian component i of cell vector a_j
 *    (the cell vectors are the COLUMNS of the 3x3 matrix), in bohr.
 *  - Real-space grid X (Sec. 2.3.1): point (i1,i2,i3) is
 *    r = i1/N1 a_1 + i2/N2 a_2 + i3/N3 a_3; arrays of grid values (potentials,
 *    densities, GMRES vectors) hold Ng = N1 N2 N3 doubles, index
 *    (i1*N2 + i2)*N3 + i3 (i3 fastest).  Their norm is the plain l2 norm of
 *    the Ng values (eq. op_discretised).
 *  - Orbital basis of k-point k (Sec. 4.1.1): all G = j1 b1 + j2 b2 + j3 b3
 *    with |k + G|^2 <= 2 Ecut, listed in lexicographic order of the signed
 *    Miller triples (j1, j2, j3); ikr_basis_millers() returns the list.
 *    The triples must satisfy -N/2 <= j < N/2 on every axis, otherwise setup
 *    fails with IKR_ERR_ARG.  Grid sizes may contain the prime factors 2, 3, 5.
 *  - Orbital vectors are complex128 (interleaved re, im), each vector stored
 *    contiguously (column-major Nb_k x nvec); coefficients are those of the
 *    normalised plane waves e_G = e^{iG.r}/sqrt(|Omega|) (Sec. 2.3.1).
 *  - All vector pointers are DEVICE pointers owned by the caller unless a
 *    parameter says "host".  The context owns copies of everything it keeps.
 *  - Every call that takes a stream enqueues its GPU work on that stream and
 *    returns after the work that produces host-visible results is complete.
 *  - Errors: every call returns an ikr_status; no exception crosses the ABI.
 *    ikr_last_error() gives a per-context message for the last failure.
 *    A failed call leaves the context usable unless it returns IKR_ERR_CUDA.
 *  - Environment: IKR_CG_FUSED=0 (read when a context first runs an FP32 CG
 *    for a given number of systems per k-point) replaces the fused CG update
 *    (one thread-block cluster per k-point, one launch per iteration) by the
 *    equivalent sequence of separate kernels; results agree to FP32 rounding.
 *    The sequence is also what runs when the fused update does not fit.
 */
#ifndef IKR_H
#define IKR_H

#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ikr_ctx ikr_ctx;

typedef enum {
  IKR_OK = 0,
  IKR_ERR_ARG = 1,       /* invalid argument (sizes, pointers, ordering) */
  IKR_ERR_CUDA = 2,      /* a CUDA runtime call failed */
  IKR_ERR_OOM = 3,       /* device allocation failed */
  IKR_ERR_NOGAP = 4,     /* eps_{Nocc+1,k} - eps_{Nocc,k} <= 0 (proof of Lemma cgtol_E needs a gap) */
  IKR_ERR_NOCONV = 5,    /* an iteration cap was reached; outputs hold the best iterate */
  IKR_ERR_NUMERIC = 6,   /* NaN/Inf or a non-positive CG curvature was detected */
  IKR_ERR_TIMEOUT = 7,   /* a wall-clock limit of the options was exceeded */
  IKR_ERR_STATE = 8      /* the call needs state the context does not have yet */
} ikr_status;

typedef enum {
  IKR_FP64 = 0,          /* every step in FP64 */
  IKR_MIXED = 1,         /* FP32 complex FFT/CG where the tolerance allows, FP64 elsewhere */
  IKR_DF64 = 2           /* ikr_apply_hamiltonian only: complex128 vectors, FP64-accurate plane
                            pass in double-float arithmetic on the FP32 units (the pass the mixed
                            path uses for its FP64-accurate sections); other calls treat it as
                            IKR_FP64 */
} ikr_precision;

/* Sternheimer CG tolerance rules (Table strategies; k-form Table strategies_k,
 * with Nocc_k N_mp replaced by Nocc = sum_k Nocc_k as the paper does). */
typedef enum {
  IKR_AGR = 0,           /* prefactor 1 */
  IKR_BAL = 1,           /* |Omega| / (2 f_nk w_k Nocc sqrt(Ng)) */
  IKR_GRT = 2,           /* sqrt|Omega| / (2 f w_k sqrt(Ng Nocc) ||Kv|| ||Re F_k^-1 Phi_k||_{2,inf}) */
  IKR_D10 = 3,           /* static tau/10 */
  IKR_D100 = 4,          /* static tau/100 */
  IKR_D10N = 5,          /* static tau/(10 ||b||) */
  IKR_GRT_EXACT = 6,     /* C_{i,nk} of Theorem inexact_gmres_dyson (App. F), gaps kept */
  IKR_FIXED = 7          /* every Sternheimer solve at opts.fixed_cg_tol */
} ikr_strategy;

/* The synthetic ground-state problem: a local potential V on the grid. */
typedef struct {
  double lattice[9];           /* cell vectors as columns, bohr */
  int dims[3];                 /* N1, N2, N3 */
  double Ecut;                 /* kinetic-energy cut-off, Ha */
  int nkpt;                    /* number of k-points */
  const double* kpoints;       /* host, nkpt x 3 fractional reciprocal coordinates */
  const double* kweights;      /* host, nkpt weights w_k (summing to 1) */
  const double* V;             /* host, Ng values of the local potential, Ha */
  double temperature;          /* Fermi-Dirac smearing T (Ha); 0 = insulator (f = 2 on N/2 bands) */
  int n_electrons;             /* N (even) */
} ikr_system;

/* Eigenpairs of H_k for every k-point (the ground state, eq. discretised_KS). */
typedef struct {
  int nbands;                  /* eigenpairs per k-point (same for all k), >= Nocc_k + 1 */
  const double* eigenvalues;   /* host, nkpt x nbands, ascending per k */
  const double* const* eigenvectors; /* host array of nkpt DEVICE pointers; entry k points to
                                        Nb_k x nbands complex128, column-major, orthonormal */
} ikr_eigenpairs;

/* Per-call statistics (N_ham of Sec. 4.1.3 counts Hamiltonian applications = CG iterations). */
typedef struct {
  int status;                  /* ikr_status of the call */
  int outer_iters;             /* GMRES steps (E applications inside the Arnoldi loop) */
  int restarts;                /* restarts of Algorithm 1 (s-update or after m steps) */
  int e_applies;               /* all E applications, restart residuals included */
  int e_applies_fp32;          /* of which ran their CG in FP32 (IKR_MIXED) */
  long long n_ham;             /* Hamiltonian applications summed over all systems */
  long long n_ham_fp64;        /* of which in FP64 */
  int cg_max_iters;            /* largest CG iteration count of a single system */
  int cg_noconv;               /* Sternheimer systems that hit the CG iteration cap */
  double est_residual;         /* final ||r~|| of GMRES */
  double sigma;                /* final s (estimate of sigma_m(H_m)) */
  double b_norm;               /* ||b|| */
  double kv_norm;              /* ||K v|| of the last E application */
  double min_cg_tol, max_cg_tol; /* range of the CG tolerances used */
  double ms;                   /* wall time of the call */
  double* history;             /* optional host array (caller-owned), receives ||r~_i|| per step */
  int history_cap;             /* its capacity; history_len <= history_cap entries are written */
  int history_len;
  double first_min_cg_tol;     /* smallest CG tolerance of the solve's first E application */
  double first_kv_norm;        /* ||K v|| of that application (the tolerance rules' ||K v_i||) */
} ikr_report;

typedef struct {
  double tau;                  /* absolute GMRES tolerance on ||b - E x|| (Algorithm 1) */
  int m;                       /* restart size m */
  int strategy;                /* ikr_strategy */
  int precision;               /* ikr_precision */
  int max_restarts;            /* cap on restarts -> IKR_ERR_NOCONV */
  int cg_maxit;                /* CG iteration cap per Sternheimer solve */
  double kerker_alpha;         /* > 0: left Kerker preconditioner T (eq. kerker), 0: off */
  double fixed_cg_tol;         /* CG tolerance of IKR_FIXED */
  double s0;                   /* initial estimate s of sigma_m(H_m) (paper: 1) */
  int use_x0;                  /* 1: x holds the initial guess x0 on input, 0: x0 = 0 */
  double timeout_s;            /* > 0: wall-clock cap -> IKR_ERR_TIMEOUT */
} ikr_solve_opts;

/* Fills opts with the paper's defaults: tau = 1e-8, m = 20, IKR_BAL, IKR_FP64,
 * max_restarts = 20, cg_maxit = 400, no Kerker, s0 = 1, x0 = 0. */
void ikr_default_opts(ikr_solve_opts* opts);

/* Creates a context for the system: enumerates the orbital bases G_k and the
 * pruned FFT geometry, uploads V, and, when eig != NULL, the ground state
 * (occupations f_nk with the Fermi level from sum_k w_k sum_n f_nk = N, eq.
 * density; N_occ,k = max{n : f_nk > 1e-10} (Sec. 2.2); the density rho and the
 * exchange kernel K^xc[rho]).  With eig == NULL only ikr_apply_hamiltonian and
 * the basis queries work until ikr_set_eigenpairs() is called.
 * Returns IKR_ERR_NOGAP for an insulator (T = 0) whose band N/2 + 1 is not above
 * band N/2 at some k-point.  *out is NULL on failure. */
ikr_status ikr_setup_groundstate(const ikr_system* sys, const ikr_eigenpairs* eig,
                                 cudaStream_t stream, ikr_ctx** out);

/* Sets or replaces the ground state of an existing context (see above). */
ikr_status ikr_set_eigenpairs(ikr_ctx* ctx, const ikr_eigenpairs* eig, cudaStream_t stream);

/* Kleinman-Bylander nonlocal part of H_k (the nonlocal term of the
 * pseudopotentials of Sec. 4, here with Gaussian projectors):
 * V_nl = sum_j D_j |beta_j><beta_j|, on each centre R_a one s and three p
 * projectors (order s, p_x, p_y, p_z) of unit norm,
 *   beta_s(r)   = (pi s^2)^-3/4 exp(-|r|^2/(2 s^2)),            s = sigma[0]
 *   beta_p,a(r) = sqrt(2)/s (pi s^2)^-3/4 r_a exp(-|r|^2/(2 s^2)), s = sigma[1]
 * (Bloch sums over the lattice), D[0] for s and D[1] for p, in Ha.
 * centres: host, ncentres x 3 Cartesian bohr; sigma, D: host, 2 each.
 * Must be called before the eigenpairs are set (IKR_ERR_STATE otherwise);
 * ncentres = 0 removes the term.  Every later H_k application (the
 * eigensolver, the CG, ikr_apply_hamiltonian) includes it; the no-allocation
 * ikr_apply_hamiltonian_noalloc then returns IKR_ERR_ARG. */
ikr_status ikr_set_nonlocal(ikr_ctx* ctx, int ncentres, const double* centres, const double* sigma, const double* D,
                            cudaStream_t stream);

/* Computes the lowest nbands eigenpairs of every H_k on the GPU and sets them
 * as by ikr_set_eigenpairs.  The ground state is the input of the method
 * (eq. discretised_KS); the paper obtains it from an SCF, which this library
 * does not run.  No counterpart in the paper's algorithms: setup only.
 * Method: Chebyshev-filtered subspace iteration with the library's own H_k
 * applications (no dense H_k), SVQB orthonormalisation and Rayleigh-Ritz; a
 * block of nbands + max(4, nbands/4) vectors, filter polynomial of the given
 * degree (>= 2), stopping when every wanted band has ||H x - theta x|| <= tol
 * (Ha, absolute) or after maxit cycles.
 * Outputs (optional, host): the eigenvalues (nkpt x nbands, ascending per k),
 * and per k-point the cycles and the final largest residual (nkpt entries).
 * Returns IKR_ERR_NOCONV (eigenpairs still set) when a k-point stopped at
 * maxit above tol; IKR_ERR_NOGAP / IKR_ERR_ARG as ikr_set_eigenpairs. */
ikr_status ikr_compute_eigenpairs(ikr_ctx* ctx, int nbands, double tol, int maxit, int degree, double* eigenvalues,
                                  int* iters, double* max_residual, cudaStream_t stream);

/* Schur-complement Sternheimer solves (Sec. 3.4.2 and Sec. 4.1.2, where the
 * paper uses them in all experiments).  enable = 1: every chi0 application
 * (ikr_apply_chi0, ikr_apply_dielectric and its adjoint, ikr_solve_response
 * and its adjoint) solves Q(H_k - eps_n)Q x = b with the extra computed bands
 * Psi_k = bands N_occ,k + 1 .. nbands of the eigenpairs split off:
 *   x = Psi a + y,  a = (lambda - eps_n)^-1 Psi^H b,  CG on R(H_k - eps_n)R y = R b,
 *   R = 1 - [Phi Psi][Phi Psi]^H,
 * which has the same solution and a larger smallest eigenvalue
 * (eps_{nbands+1} - eps_n instead of eps_{Nocc+1} - eps_n).  The terms of the
 * complement in W = R H Psi are dropped: for Rayleigh-Ritz pairs W is the
 * size of their residual.  enable = 0 restores the plain projected CG.
 * ikr_solve_sternheimer is not affected.  IKR_ERR_STATE before the eigenpairs
 * are set (setting new eigenpairs disables it again). */
ikr_status ikr_set_schur(ikr_ctx* ctx, int enable);

/* The FP32 projection products (eq. discretised_sternheimer: M = Phi^H Y, and
 * the Q-projection Y - Phi (Phi^H Y) of every FP32 CG iteration), both V_k^H Y
 * and Y - V_k C, on the 5th-generation tensor cores: tcgen05 MMAs of
 * kind::f16 on bf16 operands, every FP32 operand split exactly into three
 * bf16 pieces and six of their products accumulated in FP32 in tensor memory
 * (products as accurate as FP32 multiplications); V_k^H Y split-K over thread
 * blocks with a fixed-order reduction of the chunk partials.  mode: 0 the
 * CUDA-core kernels, 1 the tensor cores with 64-byte swizzled operand tiles,
 * 2 the tensor cores with the canonical (unswizzled) operand layout.
 * IKR_ERR_ARG for another mode; IKR_ERR_STATE before the eigenpairs are set.
 * A tensor-core launch whose internal wait runs out makes the calling solve
 * return IKR_ERR_TIMEOUT. */
ikr_status ikr_set_tensor_cores(ikr_ctx* ctx, int mode);

/* c[s][m] = <phi_m,k, y_s> for the occupied orbitals of k-point k (the
 * coefficient product of eq. discretised_sternheimer, M = Phi_k^H Y) in FP32
 * arithmetic: method 0 on the CUDA cores, 1 and 2 on the tensor cores (as
 * ikr_set_tensor_cores modes 1 and 2).  y: DEVICE, Nb_k x nvec complex64, column-major
 * (vector s at s * Nb_k); c: HOST, nvec x N_occ,k complex128 (row s).
 * IKR_ERR_ARG for a bad k, nvec < 1 or NULL pointers; IKR_ERR_TIMEOUT as above. */
ikr_status ikr_projection_coefficients(ikr_ctx* ctx, int k, int nvec, const void* y, int method, double* c,
                                       cudaStream_t stream);

/* y <- Q_k y = y - Phi_k (Phi_k^H y), the projector of eq.
 * discretised_sternheimer, in FP32 arithmetic: method 0 on the CUDA cores, 1
 * and 2 on the tensor cores (as ikr_set_tensor_cores modes 1 and 2).  y: DEVICE, Nb_k x nvec complex64, column-major,
 * overwritten.  Errors as ikr_projection_coefficients. */
ikr_status ikr_project_out(ikr_ctx* ctx, int k, int nvec, void* y, int method, cudaStream_t stream);

/* Autotuner (no counterpart in the paper).  Several kernels have variants that
 * compute the same result with different launch shapes and layouts; this call
 * times them on the context's own occupied systems (on `stream`, CUDA events,
 * best of two after one untimed run) and keeps the fastest for every later
 * call on the context:
 *   - a 4-iteration FP32 CG over all systems for each FP32 plane kernel
 *     (full-plane; compact at 4 or 5 blocks per SM) with the projection
 *     products on the CUDA cores (fused cluster update) or the tensor cores,
 *     projecting on the vector set of the context's solves (with
 *     ikr_set_schur: the occupied and the extra computed bands);
 *   - with the CUDA cores, the same CG for each cluster size of the fused
 *     update (16, 12, 10, 8 CTAs per k-point) that fits;
 *   - one FP64-accurate (double-float) H_k application over all systems for
 *     the padded and the swizzled plane kernel, on 48 x 48 planes.
 * The variants agree to FP32 (double-float) rounding.  out: HOST, 16 doubles:
 * [0..5] ms per CG iteration for (CUDA cores: plane 0, 4, 5; tensor cores:
 * plane 0, 4, 5), [6] chosen FP32 plane variant (0, 4, 5), [7] tensor cores
 * chosen (0/1), [8..9] ms of the double-float application (padded, swizzled;
 * -1 when not timed), [10] swizzled chosen (0/1), [11] chosen cluster size of
 * the fused update (0: tensor cores, no fused update), [12..15] ms per CG
 * iteration with cluster size 16, 12, 10, 8 (-1 where it does not fit).
 * IKR_ERR_STATE before the eigenpairs are set. */
ikr_status ikr_autotune(ikr_ctx* ctx, double* out, cudaStream_t stream);

/* Arithmetic throughput of the current device, measured by FMA-chain and
 * radix-4 butterfly kernels timed with CUDA events on `stream` (about 0.1 s).
 * The paper has no counterpart: these are the measured references of the ALU
 * rooflines of the plane passes, whose grid stays on chip.  out: HOST, 6
 * doubles: [0] number of SMs, [1] FP32 FMA TFLOP/s, [2] FP64 FMA TFLOP/s,
 * [3] FP32 and [4] double-float radix-4 butterflies in TFLOP/s (3 complex
 * products and 8 complex sums = 34 real flops per butterfly, a double-float
 * operation counted as one flop), [5] the device's reported SM clock in MHz.
 * IKR_ERR_ARG for NULL, IKR_ERR_CUDA if a launch fails. */
ikr_status ikr_device_peaks(double* out, cudaStream_t stream);

/* Host utility (no GPU): eigenvalues w (ascending, n) and eigenvectors v
 * (column j = eigenvector of w[j]; row-major n x n complex, interleaved) of the
 * Hermitian matrix a (row-major n x n complex, interleaved), by the cyclic
 * Jacobi rotations the eigensolver uses for its Rayleigh-Ritz steps.
 * IKR_ERR_ARG for n < 1 or NULL pointers. */
ikr_status ikr_hermitian_eigh(int n, const double* a, double* w, double* v);

/* Basis queries: number of k-points, Nb_k, and the Miller triples of G_k
 * (host output, Nb_k x 3 ints). */
int ikr_num_kpoints(const ikr_ctx* ctx);
ikr_status ikr_basis_size(const ikr_ctx* ctx, int k, int* nb);
ikr_status ikr_basis_millers(const ikr_ctx* ctx, int k, int* millers);

/* Ground-state data (host outputs, any may be NULL): occupations f (nkpt x
 * nbands), N_occ,k (nkpt), Fermi level, and the density rho (Ng doubles, DEVICE). */
ikr_status ikr_groundstate_info(const ikr_ctx* ctx, double* f, int* nocc, double* eF,
                                double* rho_device, cudaStream_t stream);

/* H_k psi for nvec vectors (eq. Hamiltonian, k-form of Sec. 4.1.1):
 *   H_k psi = |k+G|^2/2 psi + F_k (V . F_k^{-1} psi)
 * with F^{-1} = w^{-1} W^{-1} Z and F = w Z^T W (eq. fft_ifft).
 * psi, hpsi: DEVICE, Nb_k x nvec complex128 (IKR_FP64, IKR_DF64) or complex64
 * (IKR_MIXED: arithmetic in FP32).  psi and hpsi must not overlap.  IKR_ERR_ARG for a
 * grid whose Nx x Ny plane has no compiled kernel shape and does not fit in a
 * block's shared memory (the shapes compiled are 10x12, 12x12, 24x24, 32x32,
 * 40x40, 48x48 and 96x96). */
ikr_status ikr_apply_hamiltonian(ikr_ctx* ctx, int k, const void* psi, void* hpsi, int nvec,
                                 int precision, cudaStream_t stream);

/* H_k psi like ikr_apply_hamiltonian (IKR_FP64, complex128 vectors), but the
 * call allocates no device memory: no cudaMalloc, cudaFree or allocating
 * library routine.  The paper has no counterpart; this serves callers that
 * cannot allocate while they work - a stream being captured into a CUDA graph
 * (an allocation invalidates the capture), an application whose device memory
 * is owned by its own pool, a latency-bound loop that must stay out of the
 * allocator.  The context itself is created beforehand (that allocates).
 * Scratch: one static 32 MiB device array in the library, which every GPU
 * that loads the library holds until the process exits.  Each vector needs
 * 2 * 16 * N3 * ncp bytes (ncp: ncols of ikr_fft_geometry rounded up to a
 * multiple of 16); vectors are
 * processed in chunks that fit, and a grid whose single vector does not fit
 * is rejected with IKR_ERR_ARG.  The plane pass is the one
 * ikr_apply_hamiltonian runs (the compiled kernel of the grid's plane shape
 * where there is one); a grid without one whose plane does not fit in a
 * block's shared memory (about Nx, Ny > 85) is rejected with IKR_ERR_ARG, as
 * by ikr_apply_hamiltonian.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress) with that device current:
 * make that first call before any stream capture.  All calls in the process
 * share the array and its contents persist between calls; calls that overlap
 * on the GPU (other streams or threads at the same time) race on it and must
 * be serialised by the caller.  The work is enqueued on `stream`; the call
 * returns without waiting for it.  psi, hpsi: DEVICE, Nb_k x nvec complex128,
 * not overlapping. */
ikr_status ikr_apply_hamiltonian_noalloc(ikr_ctx* ctx, int k, const void* psi, void* hpsi, int nvec,
                                         cudaStream_t stream);

/* Solves the projected Sternheimer equations (eq. discretised_sternheimer)
 *   Q_k (H_k - eps_nk) Q_k x_s = Q_k rhs_s,   Q_k = 1 - Phi_k Phi_k^H,
 * for nsys systems s with k-point k_of[s] and occupied band band_of[s] (host
 * arrays; systems must be grouped by nondecreasing k), by preconditioned CG
 * from x = 0 with at least one iteration, stopping at the absolute residual
 * ||Q rhs - A x|| <= tol[s] (host array).  Iterates are kept in range(Q).
 * rhs, x: DEVICE, complex128, system s at offset s * ld where ld >= max Nb_k
 * (entries past Nb_k are ignored / left untouched).  iters_out, resid_out:
 * host arrays of nsys (may be NULL).  Returns IKR_ERR_NOCONV if a system hit
 * maxit (its x is still the last iterate). */
ikr_status ikr_solve_sternheimer(ikr_ctx* ctx, int nsys, const int* k_of, const int* band_of,
                                 const void* rhs, void* x, int ld, const double* tol, int maxit,
                                 int precision, int* iters_out, double* resid_out,
                                 cudaStream_t stream);

/* chi0 dV (eq. chi0; k-form eq. kchi0) with every Sternheimer equation solved
 * to the tolerance tol[s] (host, one per system in k-major band order, s over
 * sum_k N_occ,k; NULL: 1e-12 for all):
 *   sum_k w_k sum_n 2 f_nk Re(conj(F^-1 phi_nk) . F^-1 (dphi^P + dphi^Q)) + df_nk |F^-1 phi_nk|^2
 * dphi^P_n = sum_{m != n} f_n/(f_n^2+f_m^2) (f_n-f_m)/(eps_n-eps_m) <phi_m, dV phi_n> phi_m
 * (eq. delta_phi_P, see the design notes on its coefficient), df_n = f'_n (deps_n - deps_F).
 * dV, drho: DEVICE, Ng doubles.  report may be NULL. */
ikr_status ikr_apply_chi0(ikr_ctx* ctx, const double* dV, double* drho, const double* tol,
                          int precision, ikr_report* report, cudaStream_t stream);

/* E v = v - ||K v|| chi0(K v / ||K v||)  (eq. op_discretised), K = K^H + K^xc
 * with K^H = 4 pi/|G|^2 (G = 0 -> 0) and the LDA exchange kernel
 * K^xc = -(1/3)(3/pi)^{1/3} rho^{-2/3} (0 where rho < 1e-10).
 * tol: as in ikr_apply_chi0.  v, Ev: DEVICE, Ng doubles; may not overlap. */
ikr_status ikr_apply_dielectric(ikr_ctx* ctx, const double* v, double* Ev, const double* tol,
                                int precision, ikr_report* report, cudaStream_t stream);

/* Solves E x = b by Algorithm 1 (inexact GMRES(m) with the s-update restarts)
 * to ||b - E x|| <= tau, choosing every CG tolerance by opts->strategy
 * (Theorem inexact_gmres_dyson, Table strategies).  With kerker_alpha > 0 the
 * left-preconditioned system T E x = T b (eq. precond_dyson) is solved.
 * b, x: DEVICE, nrhs x Ng doubles; x holds x0 on input if opts->use_x0.
 * report: host array of nrhs (may be NULL).
 * nrhs > 1: the right-hand sides advance in lockstep, each with its own GMRES
 * state and tolerances; the E applications of one round share one batched CG
 * over all their Sternheimer systems, and their right-hand-side and density
 * passes are FP64-accurate (the FP32 E applications of late steps are not
 * used).  Each solution meets its own tau.  The environment variable
 * IKR_BATCH=0 solves them one after another instead.
 * Returns IKR_ERR_NOCONV (best iterate in x) if max_restarts is exceeded. */
ikr_status ikr_solve_response(ikr_ctx* ctx, int nrhs, const double* b, double* x,
                              const ikr_solve_opts* opts, ikr_report* report,
                              cudaStream_t stream);

/* Launch accounting and kernel timing (no counterpart in the paper: it
 * provides the measurements of the hot path).  Kernel classes, in order:
 *   0 z_inverse  sphere scatter + inverse z-FFT      5 cg_vector  CG vector updates
 *   1 plane      y/x FFTs, potential product, back   6 density    density accumulation
 *   2 z_forward  forward z-FFT + sphere gather       7 grid_fft   full-grid FFT passes
 *   3 proj_coef  Phi^H Y                             8 grid_ops   grid vectors, Arnoldi
 *   4 proj_apply Y - Phi C                           9 scalar     per-system scalars
 * ikr_profile_start() resets the counters; bit i of mask brackets every call
 * of class i with CUDA events on the call's stream (0: count launches only).
 * ikr_profile_read() synchronizes the context's stream and fills up to cap
 * entries (host array); it returns the number of classes. */
typedef struct {
  const char* name;            /* static class name */
  long long launches;          /* kernel launches since ikr_profile_start */
  long long timed_calls;       /* wrapper calls bracketed by events */
  double ms;                   /* summed event time of those calls */
  long long units_fp32;        /* systems processed by FP32 launches of the class */
  long long units_fp64;        /* systems processed by FP64 launches of the class */
  double ms_fp32, ms_fp64;     /* event time split by the precision of the calls */
  long long timed_calls_fp32, timed_calls_fp64;
} ikr_kernel_stat;
ikr_status ikr_profile_start(ikr_ctx* ctx, unsigned mask);
int ikr_profile_read(ikr_ctx* ctx, ikr_kernel_stat* out, int cap);
/* The pruned transform geometry (host output, 5 ints): N1, N2, N3, the number
 * of sphere columns (j1, j2) transformed along z, and of active x positions. */
ikr_status ikr_fft_geometry(const ikr_ctx* ctx, int* out);

/* The dielectric operator 1 - K chi0, the transpose of E for the symmetric chi0
 * and K (Sec. 2.2): E^T v = v - ||v|| K chi0(v/||v||).  It serves the adjoint
 * (backward) solve of a loss of drho.  Arguments as ikr_apply_dielectric. */
ikr_status ikr_apply_dielectric_adjoint(ikr_ctx* ctx, const double* v, double* Etv, const double* tol,
                                        int precision, ikr_report* report, cudaStream_t stream);

/* Solves E^T lambda = g by Algorithm 1 (the adjoint of ikr_solve_response: for
 * a loss L(drho) with drho = E^-1 chi0 dV, dL/d dV = chi0 E^-T dL/d drho).  The
 * tolerance rules are those of ikr_solve_response with ||K v_i|| replaced by
 * the bound ||K|| <= max 4 pi/|G|^2 + max |K^xc| (the Sternheimer error enters
 * through K after chi0).  Arguments as ikr_solve_response. */
ikr_status ikr_solve_response_adjoint(ikr_ctx* ctx, int nrhs, const double* g, double* lambda,
                                      const ikr_solve_opts* opts, ikr_report* report, cudaStream_t stream);

/* Frees the context and all device memory it owns.  NULL is allowed. */
void ikr_destroy(ikr_ctx* ctx);

/* Message of the last failed call on ctx ("" if none); valid until the next call. */
const char* ikr_last_error(const ikr_ctx* ctx);
/* Static name of a status code. */
const char* ikr_status_string(int status);
/* Library version string. */
const char* ikr_version(void);

#ifdef __cplusplus
}
#endif
#endif /* IKR_H */
