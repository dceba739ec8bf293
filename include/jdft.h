/*
 * jdft.h -- C ABI of the GB300 plane-wave Hamiltonian library (libjdft.so).
 *
 * The library applies the Kohn-Sham Hamiltonian of plane-wave density
 * functional theory to blocks of bands, and computes the electron density and
 * the subspace matrices, on one NVIDIA GB300 GPU.  Its operators are those of
 * the algebraic ("DFT++") formulation the JDFTx paper builds on (Sec. 2.1,
 * Software Architecture): I and J move fields between reciprocal and real
 * space by FFT, O is the overlap, diagonal in the plane-wave basis, and the
 * pseudopotential projectors (Sec. 2.2) give the nonlocal term.  The paper
 * prints no formula for them; the library uses the standard readings:
 *
 *   lattice vectors a_d = columns of R, Omega = |det R|, B = 2 pi R^{-T};
 *   FFT box S = (S0,S1,S2), N = S0 S1 S2, linear index j2 + S2 (j1 + S1 j0);
 *   basis at k: integer triples iG with (1/2)|B(iG + k)|^2 <= E_cut, ordered
 *     lexicographically by (i0, i1, i2) (k in fractional coordinates);
 *   (I X)_j = sum_G X_G exp(+2 pi i iG.j/S), (J x)_G = (1/N) sum_j x_j exp(-2 pi i iG.j/S),
 *   Idag = N J, Jdag = I / N, O = Omega;
 *   H C = Omega [ (1/2)|k+G|^2 C + J(V . I C) ] + P D P^dag C;
 *   n(r_j) += w_k sum_b f_b |(I C_b)_j|^2.
 *
 * Conventions for every call
 *   - Complex numbers are interleaved (re, im).  Precision JDFT_FP64 takes
 *     complex128 coefficient blocks; the other precisions take complex64
 *     coefficient blocks and keep V, D, densities and subspace matrices in FP64.
 *   - A coefficient block C of nb bands is band-major: band b occupies
 *     C[b*ldc .. b*ldc + npw - 1] (complex elements), ldc >= npw.
 *   - Real-space boxes are N contiguous elements per band, j2 fastest.
 *   - Pointers marked "device" are GPU global memory owned by the caller; the
 *     library only borrows them for the call.  Pointers marked "host" are
 *     ordinary host memory.  `stream` is a cudaStream_t (NULL = legacy
 *     default stream).  Compute calls are asynchronous on that stream:
 *     argument errors are reported synchronously by the return value; a
 *     kernel launch error is reported as JDFT_ERR_CUDA.
 *   - A basis handle owns device copies of its maps, potential and
 *     projectors, and a workspace that grows on demand (growth calls
 *     cudaMalloc, which synchronises the device).  One basis must not be used
 *     from two host threads at once.
 *   - On any status other than JDFT_OK, jdft_last_error() returns a message
 *     (thread-local, valid until the next call on that thread).
 */
#ifndef JDFT_H
#define JDFT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct jdft_basis_s* jdft_basis_t;

typedef enum {
    JDFT_OK = 0,
    JDFT_ERR_ARG = 1,          /* invalid argument (null pointer, size, index, alignment) */
    JDFT_ERR_CUDA = 2,         /* a CUDA runtime call or kernel launch failed */
    JDFT_ERR_OOM = 3,          /* device or host allocation failed */
    JDFT_ERR_TIMEOUT = 4,      /* a bounded device-side wait gave up */
    JDFT_ERR_NOT_POSDEF = 5,   /* overlap matrix not positive definite */
    JDFT_ERR_NOT_CONVERGED = 6,/* minimiser hit its iteration limit */
    JDFT_ERR_UNSUPPORTED = 7   /* valid request the library does not handle */
} jdft_status;

typedef enum {
    JDFT_FP64 = 0,   /* everything in FP64 */
    JDFT_FP32 = 1,   /* FFT chain in FP32, products FP32 on the CUDA cores */
    JDFT_TF32X3 = 2, /* FFT chain FP32; GEMMs as 3 TF32 tensor-core products (hi/lo split) */
    JDFT_BF16X3 = 3  /* FFT chain FP32; GEMMs as split BF16 tensor-core products */
} jdft_prec;

/* Cell and k-point description (host memory, read during jdft_basis_create only).
 *   R       row-major 3x3; column d is lattice vector a_d (bohr): R[3*i + d] = (a_d)_i
 *   S       FFT box; each S_d must be a product of 2, 3 and 5, at most 512, and
 *           at least 2*max|iG_d| + 1 over the spheres of all k-points
 *   ecut    plane-wave cutoff (Ha)
 *   nk      number of k-points (>= 1)
 *   kfrac   nk x 3, k-points in fractional reciprocal coordinates
 *   kweight nk weights w_k used by jdft_density (NULL = 1/nk each) */
typedef struct {
    double R[9];
    int S[3];
    double ecut;
    int nk;
    const double* kfrac;
    const double* kweight;
} jdft_cell_desc;

/* ---- basis ----------------------------------------------------------- */

/* Build the per-k spheres (Sec. 3, Listing 2's elec-cutoff; Sec. 2's plane-wave
 * basis) and upload the maps to the current CUDA device.  *out receives a new
 * handle that the caller releases with jdft_basis_destroy. */
jdft_status jdft_basis_create(const jdft_cell_desc* desc, jdft_basis_t* out);
jdft_status jdft_basis_destroy(jdft_basis_t basis);

/* Number of plane waves at k-point ik (the plane-wave basis, Sec. 2).  npw: host output. */
jdft_status jdft_basis_npw(jdft_basis_t basis, int ik, int* npw);

/* Sphere of k-point ik (the plane-wave basis, Sec. 2): iG (host, npw x 3, int32, row per
 * plane wave, in basis order; the caller owns it). */
jdft_status jdft_basis_gvectors(jdft_basis_t basis, int ik, int32_t* iG);

/* Scalars of the cell and grid (GridInfo, Sec. 2.1): Omega (bohr^3), N, number of (i0,i1) disk
 * columns at ik (host outputs; any may be NULL). */
jdft_status jdft_basis_info(jdft_basis_t basis, int ik, double* omega, int64_t* nbox, int* ncols);

/* ---- potential and projectors ----------------------------------------- */

/* Copy the local potential V(r_j) (device, N doubles, j2 fastest, borrowed for the call) into
 * the basis: the real-space scalar field that the Hamiltonian multiplies pointwise (Sec. 2.1,
 * Listing 1's field products).  JDFT_ERR_ARG on a null pointer. */
jdft_status jdft_set_potential(jdft_basis_t basis, const double* V, void* stream);

/* Copy the nonlocal projectors of k-point ik into the basis:
 *   P  device complex128, npw x nproj column-major (projector i at P[i*npw ..]);
 *   D  device double, nproj x nproj row-major, Hermitian (real symmetric).
 * nproj = 0 clears the nonlocal term for ik.  D is also kept as rows of its
 * nonzeros (built here, on the host: this call synchronises `stream`), so
 * that block-diagonal per-atom D costs O(nonzeros) per product.
 * (Sec. 2.2, pseudopotentials.) */
jdft_status jdft_set_projectors(jdft_basis_t basis, int ik, const void* P, int nproj,
                                const double* D, void* stream);

/* Synthetic local potential on the box (the paper has no counterpart: it stands in for the
 * pseudopotential data of the paper's workloads, Sec. 3, Listing 2):
 * V(r) = -depth sum_a sum_T exp(-|r - R_a - T|^2 / 2 width^2),
 * summed over every lattice image that comes within 10 bohr of the cell.
 * atoms: host, natoms x 3 Cartesian (bohr).  V_out: device, N doubles. */
jdft_status jdft_gaussian_potential(jdft_basis_t basis, int natoms, const double* atoms,
                                    double depth, double width, double* V_out, void* stream);

/* Synthetic projectors at k-point ik (the paper has no counterpart: they stand in for the
 * pseudopotential projectors of SpeciesInfo, Sec. 2.1): 4 per atom (s, p_x, p_y, p_z), column 4a + l,
 * P_{G,(a,l)} = F_l(k+G) exp(-i (k+G).R_a) with F_l the Fourier transform of the
 * unit-norm Gaussian-type function beta_s = N_s exp(-r^2/2 sigma^2),
 * beta_p = N_p x_l exp(-r^2/2 sigma^2).  atoms: host natoms x 3.
 * P_out: device complex128, npw x 4 natoms column-major. */
jdft_status jdft_gaussian_projectors(jdft_basis_t basis, int ik, int natoms, const double* atoms,
                                     double sigma, void* P_out, void* stream);

/* ---- algebraic operators (Sec. 2.1) ------------------------------------ */

/* psi = I C (Sec. 2.1): nb bands, C band-major (ldc), psi device nb x N complex. */
jdft_status jdft_op_I(jdft_basis_t basis, int ik, const void* C, int ldc, void* psi, int nb,
                      jdft_prec prec, void* stream);
/* C = J psi (Sec. 2.1; sphere part of the normalised forward transform). */
jdft_status jdft_op_J(jdft_basis_t basis, int ik, const void* psi, void* C, int ldc, int nb,
                      jdft_prec prec, void* stream);
/* C = Idag psi = N J psi (Sec. 2.1). */
jdft_status jdft_op_Idag(jdft_basis_t basis, int ik, const void* psi, void* C, int ldc, int nb,
                         jdft_prec prec, void* stream);
/* psi = Jdag C = I C / N (Sec. 2.1). */
jdft_status jdft_op_Jdag(jdft_basis_t basis, int ik, const void* C, int ldc, void* psi, int nb,
                         jdft_prec prec, void* stream);
/* OC = O C = Omega C (Sec. 2.1; O is diagonal in the plane-wave basis). */
jdft_status jdft_op_O(jdft_basis_t basis, int ik, const void* C, int ldc, void* OC, int ldoc,
                      int nb, jdft_prec prec, void* stream);

/* ---- the hot path ------------------------------------------------------ */

/* HC = H C for nb bands at k-point ik (kinetic + local + nonlocal terms): the
 * Kohn-Sham Hamiltonian composed from the operators of Sec. 2.1 (I, the
 * pointwise product with V, J, O) and the pseudopotential projectors of
 * SpeciesInfo (Sec. 2.1, 2.2).  C and HC must not overlap.  Scatter -> inverse
 * 3-D FFT -> x V -> forward 3-D FFT -> gather, plus kinetic and projector
 * terms.  Uses (and may grow) the basis workspace.  JDFT_ERR_ARG on null or
 * misaligned blocks, ldc/ldhc < npw, or no potential set. */
jdft_status jdft_apply_H(jdft_basis_t basis, int ik, const void* C, int ldc, void* HC, int ldhc,
                         int nb, jdft_prec prec, void* stream);

/* n_r[j] += w_ik sum_b f[b] |(I C_b)_j|^2: the electron density of ElecVars (Sec. 2.1).
 * f: device, nb doubles.  n_r: device, N doubles, accumulated (the caller zeroes it). */
jdft_status jdft_density(jdft_basis_t basis, int ik, const void* C, int ldc, const double* f,
                         int nb, double* n_r, jdft_prec prec, void* stream);

/* H C and the density of the same block in one pass over the box: HC exactly
 * as jdft_apply_H writes it, and n_r += w_ik sum_b f[b] |(I C_b)_j|^2 exactly
 * as jdft_density adds it.  The density is taken from the inverse transforms
 * I C_b that the local-potential term forms anyway (Sec. 2.1 chains
 * I -> multiply -> J; the paper computes H C and the density in separate
 * operator calls).  Arguments as for those two calls; HC and C must not
 * overlap.  Uses (and may grow) the basis workspace. */
jdft_status jdft_apply_H_density(jdft_basis_t basis, int ik, const void* C, int ldc, void* HC, int ldhc,
                                 int nb, const double* f, double* n_r, jdft_prec prec, void* stream);

/* CHC = C^dag (HC), COC = C^dag O C = Omega C^dag C: the subspace matrices of a
 * ColumnBundle for the variational minimiser (Sec. 2.1, Minimize).  Device
 * complex128 nb x nb, row-major, both triangles written, accumulated in FP64.
 * Either output may be NULL to skip it. */
jdft_status jdft_subspace(jdft_basis_t basis, int ik, const void* C, int ldc, const void* HC,
                          int ldhc, int nb, void* CHC, void* COC, jdft_prec prec, void* stream);

/* ---- orthonormalisation, subspace diagonalisation, band minimisation ----- */

/* C <- C L^{-dag} with Omega C^dag C = L L^dag, so that C^dag O C = 1 afterwards
 * (O diagonal in the plane-wave basis, Sec. 2.1).  C: device, band-major
 * (ldc >= npw), complex128 for JDFT_FP64 and complex64 otherwise; the products
 * C^dag C and C L^{-dag} run at `prec` (C^dag C accumulated in FP64), the
 * Cholesky factorisation and triangular inverse on the GPU in FP64 for every
 * precision (L^{-dag} rounded to the block type).  JDFT_CHOL_FP32=1 factors
 * FP32 blocks in FP32 instead (n <= 256: one launch of a thread-block cluster
 * sharing the matrix through distributed shared memory; JDFT_CHOL_CLUSTER=0
 * selects the multi-block path).  Uses (and may grow) the basis
 * workspace.  Synchronous.  JDFT_ERR_NOT_POSDEF if the bands are linearly
 * dependent. */
jdft_status jdft_orthonormalize(jdft_basis_t basis, int ik, void* C, int ldc, int nb, jdft_prec prec,
                                void* stream);

/* jdft_orthonormalize without the wait: the same work is queued on `stream`
 * and the factorisation's outcome is merged into the caller's device word
 * *status (max of the old value and JDFT_ERR_NOT_POSDEF on linearly dependent
 * bands, else unchanged), so a pipeline of steps can check once for all of
 * them.  U: NULL, or the overlap C^dag O C of this very block (device,
 * nb x nb row-major complex128, e.g. the COC output of jdft_subspace for the
 * same C), which is then read instead of recomputed: one iteration of the
 * minimiser forms the overlap once and uses it for both the subspace matrices
 * and the orthonormalisation (Sec. 2.1).  Returns argument and launch errors
 * only.  The paper has no such call. */
jdft_status jdft_orthonormalize_async(jdft_basis_t basis, int ik, void* C, int ldc, int nb, const void* U,
                                      jdft_prec prec, int* status, void* stream);

/* One pass of the hot path over a band block, rows a1-a9 of the method (Sec.
 * 2.1: each iteration of the band minimiser, Minimize, applies H to the
 * block, forms the subspace matrices and keeps the block O-orthonormal; the
 * density is that of ElecVars):
 *   HC = H C, n_r += w_k sum_b f_b |psi_b|^2, COC = C^dag O C, CHC = C^dag H C,
 * and with orthonormalize != 0 then C <- C L^{-dag}, where COC = L L^dag is
 * factored in FP64.  Arguments, layouts and precisions as jdft_apply_H_density
 * and jdft_subspace (C, HC: band-major blocks of nb rows, leading dimensions
 * ldc, ldhc >= npw; f: device nb FP64; n_r: device box, accumulated; CHC, COC:
 * device nb x nb complex128, overwritten).  Differences from the separate
 * calls: COC is formed from the input block first, and its factorisation runs
 * on a second stream owned by the basis while H C is applied (a few SMs are
 * left to it), joining `stream` before C is rotated; the BF16x3 products
 * share one BF16 split of C.  status: device int (required with
 * orthonormalize), raised to JDFT_ERR_NOT_POSDEF if the overlap is not
 * positive definite; it is never cleared.  Asynchronous on `stream`; grows the
 * basis workspaces (synchronously) on first use.  Returns argument and launch
 * errors.  Calls for the same basis must not overlap on the GPU. */
jdft_status jdft_hamiltonian_step(jdft_basis_t basis, int ik, void* C, int ldc, void* HC, int ldhc, int nb,
                                  const double* f, double* n_r, void* CHC, void* COC, int orthonormalize,
                                  int* status, jdft_prec prec, void* stream);

/* Eigenvalues (ascending) of a Hermitian nb x nb matrix A (device complex128,
 * row-major), by cyclic Jacobi rotations in FP64 on the GPU; eigs: device,
 * nb doubles.  Synchronous.  The subspace diagonalisation that gives the band
 * energies from C^dag H C in the minimiser (Sec. 2.1, Minimize). */
jdft_status jdft_subspace_eigs(int nb, const void* A, double* eigs, void* stream);

/* Learned per-coefficient preconditioner for the band minimiser (the paper
 * has no counterpart; it stands in for the Teter preconditioner, Teter, Payne
 * & Allan, PRB 40, 12255 (1989)): a 3 -> 64 -> 64 -> 1 network, SiLU
 * hidden activations, softplus output (so K > 0).  Parameters, 4481 floats in
 * this order: W1 (64x3 row-major), b1 (64), W2 (64x64), b2 (64), W3 (64), b3 (1).
 * Features per coefficient G of band b: x = (1/2)|k+G|^2 / T_b,
 * log(1 + T_b), (h_b - min_b h_b) / T_b, with T_b the band kinetic energy and
 * h_b = (C^dag H C)_bb the band's Rayleigh quotient. */
typedef struct jdft_mlp_s* jdft_mlp_t;

/* Create a network from 4481 host floats (copied; the caller keeps ownership
 * of params).  The network keeps an FP32 master copy, the BF16 copy its
 * kernels compute with, and Adam moments. */
jdft_status jdft_mlp_create(const float* params, jdft_mlp_t* out);
jdft_status jdft_mlp_destroy(jdft_mlp_t mlp);
/* Copy the FP32 master parameters to host memory (4481 floats). */
jdft_status jdft_mlp_get_params(jdft_mlp_t mlp, float* params);
/* K for `rows` feature triples: feats device float rows x 3, K device float rows. */
jdft_status jdft_mlp_forward(jdft_mlp_t mlp, int64_t rows, const float* feats, float* K, void* stream);
/* Loss and gradient over training rows (device float rows x 5: f1, f2, f3, a, q):
 * loss = sum (K^2 a - 2 K q) / sum a.  grad: device float 4481 (overwritten);
 * loss: device double[2] (loss, sum a; overwritten). */
jdft_status jdft_mlp_loss_grad(jdft_mlp_t mlp, int64_t rows, const float* data, float* grad,
                               double* loss, void* stream);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) with a device gradient. */
jdft_status jdft_mlp_adam_step(jdft_mlp_t mlp, const float* grad, float lr, void* stream);
/* Training rows from a minimiser snapshot C (device complex128, nb bands,
 * ld = npw) and the converged block Cstar: for coefficients
 * i = offset + r*stride of the band-major block, (f1, f2, f3, |R|^2, Re(conj(R) t))
 * with R = H C - O C (C^dag H C) and t = C - Cstar (Cstar^dag O C); the q
 * column is then scaled by sum(a)/sum(q) over the emitted rows, so the best
 * constant K is 1 (the minimiser's line step makes the overall scale of the
 * preconditioner irrelevant; this keeps targets of different cells and
 * iterations on one scale).  rows_out = NULL only returns the row count in
 * *nrows.  Synchronous. */
jdft_status jdft_mlp_rows(jdft_basis_t basis, int ik, const void* C, const void* Cstar, int nb,
                          int64_t stride, int64_t offset, float* rows_out, int64_t* nrows,
                          void* stream);

typedef enum {
    JDFT_PRECOND_IDENTITY = 0,
    JDFT_PRECOND_TETER = 1,   /* Teter, Payne & Allan, PRB 40, 12255 (1989) */
    JDFT_PRECOND_MLP = 2      /* the learned network (opts.mlp) */
} jdft_precond;

typedef struct {
    double tol;             /* stop when ||H C - O C (C^dag H C)||_F / sqrt(Omega) < tol (Ha) */
    int max_iter;           /* iteration limit over all phases */
    jdft_precond precond;
    jdft_prec prec;         /* JDFT_FP64, or a mixed mode for the bulk iterations */
    double switch_tol;      /* mixed modes: promote to FP64 below this residual (0 = 1e-4) */
    double occupation;      /* f per band (0 = 2) */
    jdft_mlp_t mlp;         /* weights for JDFT_PRECOND_MLP, else NULL */
} jdft_min_opts;

typedef struct {
    int iterations;         /* CG iterations, all phases */
    int mixed_iterations;   /* of which in the mixed-precision phase */
    int converged;
    double energy;          /* f tr(C^dag H C) at exit (Ha) */
    double residual;        /* the stopping residual at exit (Ha) */
    double seconds;         /* wall time of the call */
    int precond_fallback;   /* 1: the learned preconditioner failed a check (a non-finite or non-descent
                               direction, no energy decrease along it, or 40 iterations without progress)
                               and Teter's took over for the rest of the call */
} jdft_min_report;

/* Preconditioned all-band conjugate-gradient minimisation of E = f tr(C^dag H C)
 * over O-orthonormal C at fixed potential (Sec. 2.1 Minimize; Sec. 2.2).
 * C: device complex128 band-major, in: starting guess (any linearly
 * independent block), out: converged orthonormal block.  eigs: device nb
 * doubles (NULL to skip): eigenvalues of C^dag H C at exit.  report: host.
 * Synchronous.  Allocates its working blocks for the duration of the call.
 * JDFT_ERR_NOT_CONVERGED (with C and report filled) if max_iter is reached. */
jdft_status jdft_minimize_bands(jdft_basis_t basis, int ik, void* C, int ldc, int nb,
                                const jdft_min_opts* opts, double* eigs, jdft_min_report* report,
                                void* stream);

/* ---- self-consistent field (Sec. 2.1: Coulomb, ExCorr, Pulay; Sec. 2.2) ---
 * Real-space fields here are real FP64 boxes of N values (device, j2 fastest).
 * The full-box transforms use a complex FP64 box of the basis (16 N bytes plus
 * 1 MB of partial sums, grown synchronously on first use); calls on the same
 * basis must not overlap on the GPU.  Energies go to device doubles, summed in
 * a fixed order (deterministic). */

/* Hartree potential of the density n (the periodic Coulomb kernel of class
 * Coulomb, Sec. 2.1): with nt = J n over the whole box (frequencies folded to
 * [-S/2, S/2) per axis, G = B iG),  V_H = I (4 pi nt(G) / |G|^2), the G = 0 term
 * dropped (a uniform neutralising background).  vh: device N doubles, must not
 * overlap n.  energy: device double or NULL; receives
 * E_H = (Omega/2) sum_G 4 pi |nt(G)|^2 / |G|^2.  Asynchronous. */
jdft_status jdft_hartree(jdft_basis_t basis, const double* n, double* vh, double* energy, void* stream);

/* Local-density exchange-correlation (class ExCorr, Sec. 2.1; LDA among the
 * semilocal functionals of Sec. 2.2), spin-unpolarised: Slater exchange plus
 * the Perdew-Zunger 1981 fit (PRB 23, 5048) of the Ceperley-Alder correlation.
 * Points with n <= 0 get e_xc = v_xc = 0.  vxc: device N doubles (NULL to skip;
 * may be n itself); energy: device double or NULL, receives
 * E_xc = (Omega/N) sum_j n_j e_xc(n_j).  Asynchronous. */
jdft_status jdft_xc_lda(jdft_basis_t basis, const double* n, double* vxc, double* energy, void* stream);

/* Kohn-Sham potential V_KS = V_ion + V_H[n] + v_xc[n] in one Hartree chain,
 * the potential and exchange-correlation terms added in the last transform's
 * epilogue.  vks: device N doubles, overlapping neither n nor vion.  energies:
 * device double[2] or NULL, receives (E_H, E_xc) as jdft_hartree and
 * jdft_xc_lda define them.  Asynchronous. */
jdft_status jdft_ks_potential(jdft_basis_t basis, const double* n, const double* vion, double* vks,
                              double* energies, void* stream);

/* Pulay mixing of densities ("self-consistency by Pulay mixing", class Pulay,
 * Sec. 2.1; P. Pulay, Chem. Phys. Lett. 73, 393 (1980)).  The mixer keeps the
 * last `history` pairs (n_in^i, R^i = n_out^i - n_in^i) on the device (2 x history
 * x n doubles, allocated by jdft_pulay_create).  A step stores the new pair,
 * finds c minimising |sum_i c_i R^i| (plain sum over the box) subject to
 * sum_i c_i = 1 from the bordered system [A 1; 1^T 0][c; lam] = [0; 1],
 * A_ij = <R^i, R^j> (Gaussian elimination with partial pivoting in FP64 on the
 * GPU; while a pivot falls below 1e-13 max |A_ii| the oldest pair is dropped),
 * and writes n_next = sum_i c_i (n_in^i + alpha R^i). */
typedef struct jdft_pulay_s* jdft_pulay_t;

/* n: values per density (>= 1); history in [1, 16]; alpha in (0, 1].  Uses the
 * current device.  JDFT_ERR_OOM if the history does not fit. */
jdft_status jdft_pulay_create(int64_t n, int history, double alpha, jdft_pulay_t* out);
jdft_status jdft_pulay_destroy(jdft_pulay_t mixer);
/* Forget the stored pairs (the next step is plain linear mixing). */
jdft_status jdft_pulay_reset(jdft_pulay_t mixer);
/* One mixing step: n_in, n_out, n_next device n doubles; n_next may be n_in,
 * not n_out.  Asynchronous on `stream`; steps of one mixer must be issued in
 * order from one host thread. */
jdft_status jdft_pulay_step(jdft_pulay_t mixer, const double* n_in, const double* n_out, double* n_next,
                            void* stream);
/* Number of pairs the last step combined (host int; waits for `stream`); a
 * diagnostic the paper has no counterpart for. */
jdft_status jdft_pulay_used(jdft_pulay_t mixer, int* used, void* stream);

typedef struct {
    double tol_energy;      /* converged when |E - E_prev| < tol_energy (Ha; 0 = 1e-8) ... */
    double tol_density;     /* ... and sqrt((Omega/N) sum_j (n_out - n_in)_j^2) < tol_density (0 = 1e-6) */
    int max_iter;           /* SCF iterations (0 = 100) */
    int history;            /* Pulay pairs kept (0 = 8, at most 16) */
    double alpha;           /* Pulay mixing fraction (0 = 0.5) */
    double band_tol;        /* band minimiser tolerance of the converged iterations (0 = 1e-9) */
    int band_max_iter;      /* band minimiser iteration limit (0 = 1000) */
    jdft_precond precond;   /* band minimiser preconditioner */
    jdft_prec prec;         /* band minimiser precision schedule (JDFT_FP64 or a mixed mode) */
    double occupation;      /* f per band (0 = 2) */
    jdft_mlp_t mlp;         /* weights for JDFT_PRECOND_MLP, else NULL */
    double band_tol_factor; /* iteration i solves the bands to max(band_tol, factor x the density residual
                               of iteration i - 1), the first to max(band_tol, 1e-3): loose solves while
                               the density is far from self-consistent (0 = 0.01; < 0: band_tol always) */
} jdft_scf_opts;

typedef struct {
    int iterations;         /* SCF iterations taken */
    int converged;
    int band_iterations;    /* band CG iterations, all SCF iterations and k-points */
    int band_unconverged;   /* band solves that stopped at band_max_iter */
    double energy;          /* total energy E (Ha) of the last iteration */
    double band_energy;     /* sum_k w_k f sum_b eps_kb */
    double double_counting; /* -(Omega/N) sum_j n_out,j (V_H + v_xc)[n_in]_j */
    double hartree;         /* E_H[n_out] */
    double xc;              /* E_xc[n_out] */
    double residual;        /* density residual of the last iteration */
    double seconds;         /* wall time of the call */
} jdft_scf_report;

/* Self-consistent field loop at fixed occupations (Sec. 2.2: SCF by Pulay
 * mixing, the alternative to total-energy minimisation).  The electrons see
 * V_KS[n] = V_ion + V_H[n] + v_xc[n] (jdft_ks_potential); the basis's projectors
 * stay as set.  C: host array of nk device pointers, one complex128 band-major
 * block of nb bands per k-point (ldc >= npw of every k), in: starting guess,
 * out: the orbitals of the last iteration (O-orthonormal).  vion: device N
 * doubles.  The start density is that of the orthonormalised starting blocks.
 * Each iteration: V_KS of the input density -> jdft_minimize_bands at every
 * k-point (warm-started, to the tolerance band_tol_factor sets) -> output
 * density n_out -> total energy
 *   E = sum_k w_k f sum_b eps_kb - (Omega/N) sum_j n_out,j (V_H + v_xc)[n_in]_j
 *       + E_H[n_out] + E_xc[n_out]
 * -> convergence test (both tolerances, from the second iteration) -> Pulay step.
 * n_r: device N doubles, receives n_out of the last iteration; eigs: device
 * nk x nb doubles or NULL, the last band energies.  On return the basis holds
 * V_KS of the last input density as its potential.  report: host.  Synchronous;
 * allocates its working fields (4 N doubles), the mixer and the minimiser's
 * blocks for the duration of the call.  JDFT_ERR_NOT_CONVERGED (outputs and
 * report filled) if max_iter is reached. */
jdft_status jdft_scf(jdft_basis_t basis, void* const* C, int ldc, int nb, const double* vion, double* n_r,
                     double* eigs, const jdft_scf_opts* opts, jdft_scf_report* report, void* stream);

/* ---- spinor bands (noncollinear magnetism, Sec. 2.2; ColumnBundle, Sec. 2.1)
 * A spinor block of nb bands is 2 nb coefficient rows of a band-major block:
 * row 2b holds band b's up component, row 2b + 1 its down component (same
 * sphere, ldc >= npw).  The local potential is V 1 + M . sigma: V is the
 * basis potential (jdft_set_potential), M a real 3-vector field given per
 * call as device 3 x N doubles (M_x, then M_y, then M_z).  Pauli matrices
 * sigma_x = [[0,1],[1,0]], sigma_y = [[0,-i],[i,0]], sigma_z = [[1,0],[0,-1]].
 * JDFT_FP64 (complex128 blocks), or JDFT_FP32, JDFT_TF32X3, JDFT_BF16X3 (complex64
 * blocks, FP32 transforms; the precision selects the projector products as in
 * jdft_apply_H).
 * Both calls use a spinor workspace of the basis, grown synchronously, besides
 * the one jdft_apply_H / jdft_op_I use: for FP32 blocks on boxes of 128 x 128
 * (or 16 x 12) planes, the fused chain's column buffer (up to 512 MB of
 * component rows) and M in FP32; otherwise the real-space boxes of a chunk of
 * bands (at most 256 MB) plus the chunk's sphere rows. */

/* HC = H C for nb spinor bands: the scalar Hamiltonian of jdft_apply_H on
 * every component row, plus Omega J((M . sigma) I C) coupling each band's two
 * components (on the fused path the 2 x 2 product V + M . sigma replaces the
 * multiply by V inside the plane pass).  C, HC must not overlap (ldhc >= npw).
 * Asynchronous. */
jdft_status jdft_apply_H_spinor(jdft_basis_t basis, int ik, const double* M, const void* C, int ldc, void* HC,
                                int ldhc, int nb, jdft_prec prec, void* stream);

/* n_r[j] += w_ik sum_b f_b (|psi_up|^2 + |psi_dn|^2) and the magnetisation
 * m_r[c N + j] += w_ik sum_b f_b psi^dag sigma_c psi (c = x, y, z), psi = I C.
 * f: device nb doubles; n_r: device N doubles; m_r: device 3 N doubles (both
 * accumulated; the caller zeroes them).  Asynchronous. */
jdft_status jdft_density_spinor(jdft_basis_t basis, int ik, const void* C, int ldc, const double* f, int nb,
                                double* n_r, double* m_r, jdft_prec prec, void* stream);

/* ---- augmented overlap (ultrasoft pseudopotentials, Sec. 2.2; O, Sec. 2.1) --
 * With augmentation charges Q on the projectors of the nonlocal term, the
 * overlap of coefficient blocks is S C = Omega C + P Q P^dag C and band
 * energies are the eigenvalues of the pencil (C^dag H C, C^dag S C).  Only
 * the calls of this section use Q; jdft_op_O, jdft_subspace, the
 * orthonormalisation, jdft_hamiltonian_step and jdft_minimize_bands keep the
 * plain O = Omega; jdft_minimize_bands_generalized solves the generalised
 * problem. */

/* Set (Q: device nproj x nproj doubles, row-major, symmetric; copied) or clear
 * (Q = NULL) the augmentation of k-point ik's projectors.  Needs the
 * projectors (jdft_set_projectors, which also clears Q).  Q is kept dense and
 * as rows of its nonzeros (built on the host: synchronises `stream`).
 * JDFT_ERR_ARG if Q is not symmetric or no projectors are set. */
jdft_status jdft_set_augmentation(jdft_basis_t basis, int ik, const double* Q, void* stream);

/* SC = S C = Omega C + P Q P^dag C for nb bands (band-major blocks, ldc, ldsc >=
 * npw, not overlapping), through the same projector products and precisions
 * as the nonlocal term of jdft_apply_H (complex128 for JDFT_FP64, complex64
 * otherwise).  Without augmentation SC = Omega C.  May grow the basis
 * workspace.  Asynchronous. */
jdft_status jdft_op_S(jdft_basis_t basis, int ik, const void* C, int ldc, void* SC, int ldsc, int nb,
                      jdft_prec prec, void* stream);

/* Generalised subspace matrices of an FP64 block: CHC = C^dag (HC), CSC =
 * C^dag S C (device complex128 nb x nb row-major, overwritten), and with eigs
 * (device nb doubles, or NULL) the eigenvalues of the pencil (CHC, CSC),
 * ascending: C^dag S C = L L^dag factored in FP64, then the eigenvalues of
 * L^{-1} CHC L^{-dag} by cyclic Jacobi rotations (generalised Rayleigh-Ritz).
 * C, HC: complex128 band-major (ldc, ldhc >= npw).  Synchronous; allocates
 * its scratch (three blocks) for the call.  JDFT_ERR_NOT_POSDEF if C^dag S C
 * is not positive definite. */
jdft_status jdft_subspace_generalized(jdft_basis_t basis, int ik, const void* C, int ldc, const void* HC,
                                      int ldhc, int nb, void* CHC, void* CSC, double* eigs, void* stream);

/* C <- C L^{-dag} with C^dag S C = L L^dag (FP64), so that C^dag S C = 1
 * afterwards.  C: complex128 band-major.  Synchronous; allocates its scratch
 * for the call.  JDFT_ERR_NOT_POSDEF on linearly dependent bands. */
jdft_status jdft_orthonormalize_generalized(jdft_basis_t basis, int ik, void* C, int ldc, int nb, void* stream);

/* Lowest nb states of the generalised problem H c = e S c by all-band
 * preconditioned conjugate gradients (Sec. 2.1 Minimize; the norm-conserving
 * jdft_minimize_bands with S in place of Omega): C kept S-orthonormal; gradient
 * G = H C - S C (C^dag H C); Teter or identity preconditioner; Polak-Ribiere
 * directions made S-orthogonal to C; second-order line step halved while the
 * energy of the S-orthonormalised trial block rises by more than 64 FP64 ulp;
 * converged when ||G||_F / sqrt(Omega) < opts->tol.  FP64 only (opts->prec =
 * JDFT_FP64); opts->switch_tol and opts->mlp are not used.  C: device
 * complex128 band-major, in: start, out: converged S-orthonormal block.  eigs:
 * device nb doubles or NULL.  report: host (iterations, energy f tr C^dag H C,
 * residual, seconds).  Synchronous; allocates its working blocks for the call.
 * JDFT_ERR_NOT_CONVERGED (with C and report filled) at max_iter. */
jdft_status jdft_minimize_bands_generalized(jdft_basis_t basis, int ik, void* C, int ldc, int nb,
                                           const jdft_min_opts* opts, double* eigs, jdft_min_report* report,
                                           void* stream);

/* ---- scalar fields and the linear dielectric (Sec. 2.1, Listing 1) --------
 * A reciprocal-space field (ScalarFieldTilde) is a full complex128 box X(G) of
 * N values (device, j2 fastest), slot iG mod S holding G = B iG with
 * frequencies folded to [-S/2, S/2) per axis.  A real-space field
 * (ScalarField) is a box of N values; these calls take it as complex128. */

/* x = I X: x_j = sum_G X(G) exp(+i G.r_j) over the whole box (Sec. 2.1, I on
 * scalar fields).  X and x may be the same buffer.  FP64.  Asynchronous. */
jdft_status jdft_field_I(jdft_basis_t basis, const void* X, void* x, void* stream);
/* X = J x: X(G) = (1/N) sum_j x_j exp(-i G.r_j) (Sec. 2.1, J on scalar fields).
 * x and X may be the same buffer.  FP64.  Asynchronous. */
jdft_status jdft_field_J(jdft_basis_t basis, const void* x, void* X, void* stream);

/* The dielectric operator of the paper's LinearPCM example (Sec. 2.1,
 * Eq. (Poisson), Listing 1's hessian):
 *   out~ = -(1/4 pi) div J(eps * I(grad phi~)),  grad = i G_d, div = sum_d i G_d,
 * Hermitian and positive semi-definite for eps > 0, zero on G = 0.  eps: device
 * N doubles (real space); phi_t, out_t: device complex128 reciprocal-space boxes
 * that must not overlap.  Uses the basis field workspace (three complex boxes
 * and 1 MB, grown synchronously on first use).  Asynchronous. */
jdft_status jdft_pcm_hessian(jdft_basis_t basis, const double* eps, const void* phi_t, void* out_t,
                             void* stream);

typedef struct {
    int iterations;         /* CG iterations (one hessian each; FP32 ones for JDFT_FP32) */
    int converged;
    double residual;        /* |r| / |rho~| at exit, r = rho~ - hessian(phi~) in FP64 (plain sums, G != 0) */
    double A_diel;          /* (1/2) Re sum_G conj(phi~ - 4 pi rho~ / G^2) Omega rho~ (Ha) */
    double seconds;         /* wall time of the call */
    int fp64_hessians;      /* FP64 hessians applied (= iterations for JDFT_FP64) */
} jdft_pcm_report;

/* Solve -4 pi rho = div(eps grad phi) for phi~ by preconditioned conjugate
 * gradients on reciprocal-space fields (Sec. 2.1, class LinearSolvable; the
 * paper's Listing 1 `solve(rhoTilde)`), then the solvation energy of
 * Eq. (Adiel) (`getAdiel`).  The G = 0 term of rho~ is ignored (a neutral
 * charge) and phi~(0) = 0.  Preconditioner: the Coulomb kernel 4 pi / G^2 (the
 * exact inverse for eps = 1).  Start phi~ = 0; converged when
 * |r| <= tol |rho~|, r = rho~ - hessian(phi~).
 *   prec JDFT_FP64: CG in FP64 throughout.
 *   prec JDFT_FP32: the same CG run in FP32 (fields, transforms and eps in
 *     FP32, sums in FP64) on the correction e, with reliable updates (the
 *     paper fixes no precision): whenever the FP32 residual has fallen by 1e-4
 *     since the last update, or below tol |rho~| / 2, e is added to phi~ in FP64
 *     and the residual is
 *     replaced by r = rho~ - hessian(phi~) from one FP64 hessian (the search
 *     direction kept); it stops at the same tolerance on that FP64 residual,
 *     or when an update no longer lowers it.
 * eps: device N doubles (> 0); rho_t, phi_t: device complex128 boxes (phi_t
 * overwritten, not overlapping rho_t).  max_iter: limit on CG iterations (all
 * rounds).  report: host.  Synchronous (one host read of the residual per
 * iteration); uses the basis field workspace (JDFT_FP64: six complex128
 * boxes; JDFT_FP32: ten; and 1 MB).  JDFT_ERR_NOT_CONVERGED (phi_t and report
 * filled) if the tolerance is not reached. */
jdft_status jdft_pcm_solve(jdft_basis_t basis, const double* eps, const void* rho_t, void* phi_t, double tol,
                           int max_iter, jdft_prec prec, jdft_pcm_report* report, void* stream);

/* ---- schedule autotuning (the paper has no counterpart) ------------------ */

/* Time jdft_apply_H on the caller's blocks for band-chunk budgets of
 * 32 ... 1024 MB (the column buffer passed between the chain kernels; small
 * chunks stay in L2, large ones make fewer launches; default 256 MB) and keep
 * the fastest in the basis for later calls.
 * Overwrites HC.  *chunk_mb (host, may be NULL) receives the choice.
 * Synchronous; may grow the workspace. */
jdft_status jdft_autotune_chunk(jdft_basis_t basis, int ik, const void* C, int ldc, void* HC, int ldhc,
                                int nb, jdft_prec prec, int* chunk_mb, void* stream);

/* Split-K schedule of the tensor-core product out = A^dag B (M x N over K;
 * A: M rows of K, B: N rows of K, device complex64, row strides lda, ldb):
 * times the default split count and multiples of it (never fewer splits than
 * keep <= 4096 complex K per block accumulating in tensor memory) and keeps
 * the fastest for this (M, N, K, operand type) in a process-wide table that
 * later products of that shape use.  prec JDFT_TF32X3 or JDFT_BF16X3 (other
 * precisions have no schedule: *splits = 0).  *splits (host, may be NULL)
 * receives the choice.  Synchronous; allocates an M x N scratch. */
jdft_status jdft_autotune_gemm(int M, int N, int K, const void* A, int lda, const void* B, int ldb,
                               jdft_prec prec, int* splits, void* stream);

typedef struct {
    int chunk_mb;          /* band-chunk budget kept for the chain kernels */
    int splits_subspace;   /* split-K count kept for the nb x nb x npw products (0: no schedule) */
    int splits_projector;  /* the same for the nproj x nb x npw projection P^dag C (0: none) */
    int plane_bands;       /* bands per plane-pass work item kept for FP32 blocks: 2 (band pairs,
                              packed FP32) or 1; 0 when the box has no band-pair kernel */
} jdft_tune_report;

/* Autotune everything the Hamiltonian, density and subspace calls of this
 * block use: the band-chunk budget of the FFT chain (jdft_autotune_chunk),
 * the plane pass's work-item shape for FP32 blocks (one band or a band pair
 * per (plane, item), where both are compiled; kept in the basis) and the
 * split-K schedules of the block's subspace and projector products
 * (jdft_autotune_gemm).  Overwrites HC.  Synchronous; may grow the workspace. */
jdft_status jdft_autotune(jdft_basis_t basis, int ik, const void* C, int ldc, void* HC, int ldhc, int nb,
                          jdft_prec prec, jdft_tune_report* report, void* stream);

/* ---- batches in one CUDA graph ------------------------------------------ */
/* The paper distributes k-points over MPI processes (Sec. 3); here a batch of
 * k-points or of independent cells runs from one graph launch on one GPU. */

/* One Hamiltonian application of a batch: H C for nb bands of k-point ik of
 * `basis` (arguments as for jdft_apply_H; device buffers owned by the caller). */
typedef struct {
    jdft_basis_t basis;
    int ik;
    const void* C;
    int ldc;
    void* HC;
    int ldhc;
    int nb;
    jdft_prec prec;
} jdft_apply_item;

typedef struct jdft_batch_s* jdft_batch_t;

/* Record the n applications (host array, copied) as one CUDA graph: each item
 * runs once (warm-up, on a private stream; its HC is written), then all are
 * captured in order and instantiated.  The k-points of one cell (uneven sphere
 * sizes) and independent cells with their own boxes can be mixed.  The graph
 * keeps the given device pointers: keep the buffers alive, refill the C blocks
 * as needed, and replay with jdft_batch_launch.  Items that share a basis share
 * its workspace and run in order; a replay must not overlap other calls on the
 * same bases.  Synchronous: waits for all earlier work on the device first. */
jdft_status jdft_batch_create(int n, const jdft_apply_item* items, jdft_batch_t* out);
/* Replay every application of the batch on `stream` with one graph launch. */
jdft_status jdft_batch_launch(jdft_batch_t batch, void* stream);
jdft_status jdft_batch_destroy(jdft_batch_t batch);
/* 1 if the batch runs its FFT chain k-batched: all items are k-points of one
 * basis with FP32 blocks on a box the band-pair kernels serve (128 x 128
 * planes), so each chain stage is one launch over all items (each item with
 * its own sphere maps and a column buffer the batch owns); else 0 (one
 * jdft_apply_H per item in the graph).  The paper has no counterpart. */
int jdft_batch_is_kbatched(jdft_batch_t batch);

/* ---- the Hamiltonian without device allocation --------------------------- */

/* Same result as jdft_apply_H (same arguments, layouts and precisions), but the
 * call allocates no device memory.  The paper has no counterpart: this exists
 * for callers that cannot let the library call cudaMalloc -- applications that
 * own a fixed device-memory budget or a pool allocator that must account for
 * every device byte, and latency-critical loops where a synchronising
 * allocation is unacceptable.
 *
 * The intermediate column buffer and the projector products live in one static
 * 32 MiB device array inside libjdft.so, which every GPU that loads the library
 * holds until the process exits.  Bands are processed in chunks that fit it;
 * if a single band of this basis needs more than 32 MiB
 * (S2 x ncols x element size + nproj x (16 + element size) bytes), the call
 * returns JDFT_ERR_ARG and the caller should use jdft_apply_H.
 *
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) and caches it; make that first call before any stream
 * capture.  Every call shares the one array: calls whose work overlaps on the
 * GPU (different streams, or different host threads) race on it and must be
 * serialised by the caller.  The basis must already hold its potential and
 * projectors (jdft_set_potential / jdft_set_projectors). */
jdft_status jdft_apply_H_noalloc(jdft_basis_t basis, int ik, const void* C, int ldc, void* HC,
                                 int ldhc, int nb, jdft_prec prec, void* stream);

/* ---- diagnostics and tracing (the paper has no counterpart) ------------ */

/* Turn per-kernel timing on (1) or off (0).  While on, every kernel launch of
 * the library is bracketed by two CUDA events recorded on its stream. */
jdft_status jdft_profile_enable(int on);

/* Wait for the recorded events and write one line per kernel name,
 * "name launches total_ms\n", into buf (host, buflen bytes, NUL-terminated);
 * then forget the records.  JDFT_ERR_ARG if buf is too small. */
jdft_status jdft_profile_read(char* buf, int buflen);

/* Wait for `stream`, then report JDFT_ERR_TIMEOUT if a bounded device-side wait
 * (the tensor-core products' barrier waits) gave up since the last call, and
 * clear the record.  JDFT_OK otherwise. */
jdft_status jdft_device_status(void* stream);

/* Limit, in seconds, of each device-side wait of the tensor-core products on
 * the current device (default 2 s; kernels launched after the call use it).
 * A wait that runs out records JDFT_ERR_TIMEOUT for jdft_device_status, stops
 * issuing products, waits (under a fixed 2 s limit of its own) for the products
 * it already committed, and frees its tensor memory; the product's output is
 * then incomplete.  0 makes every such product give up at its first wait,
 * which tests of the failure path use.  JDFT_ERR_ARG outside [0, 60].  The
 * paper has no counterpart. */
jdft_status jdft_set_wait_limit(double seconds);

/* Measured FP32 arithmetic peak of the current device, in TFLOP/s: chains of
 * scalar fused multiply-adds (*ffma_tflops) and of packed two-wide ones
 * (*ffma2_tflops) on every SM, timed with CUDA events on `stream` (best of
 * three after one untimed launch); *sms receives the device's SM count.  All
 * three outputs are host pointers.  Synchronous, about 0.1 s.  This is the
 * denominator of the FFT kernels' arithmetic roofline; the paper has no
 * counterpart. */
jdft_status jdft_measure_fp32_peak(double* ffma_tflops, double* ffma2_tflops, int* sms, void* stream);

/* Number of kernels the library has launched in this process (all calls).
 * Diagnostics calls have no counterpart in the paper. */
long long jdft_launch_count(void);


/* Message of the last non-OK status on this thread ("" if none). */
const char* jdft_last_error(void);

/* Library version string. */
const char* jdft_version(void);

#ifdef __cplusplus
}
#endif

#endif /* JDFT_H */
