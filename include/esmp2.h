/* esmp2.h -- C ABI of the GB300 (sm_103a) ESMP2-TOP(1) library.
 *
 * ESMP2 (excited-state-specific second-order perturbation theory) corrects an
 * excited-state mean-field (ESMF) reference Psi0 = sum_ia C_ia (a+_a a_i + a+_a a_i)|Phi>
 * (singlet, closed-shell coefficient zero; Sec. II.A, Eq. psi0).  The library
 * works in the transition-orbital-pair (TOP) basis of Sec. II.A (SVD C = U Lambda V^+,
 * Eqs. 2-4) and solves the first-order equation
 *        (H0 - E0) |Psi1> = -Q H |Psi0>                     (Sec. II.C-D)
 * with the modified zeroth-order Hamiltonian of Eq. qfq_replacement: the Fock
 * operator F acts fully on the doubles (D) and on the L-triples (triples holding
 * the large transition-orbital pair t -> t', TOP(1)), and only through its diagonal
 * on the S- and N-triples, which are therefore inverted directly.  E2 = <Psi0|H|Psi1>.
 *
 * Conventions shared by every call
 *  - No exceptions cross the ABI; every call returns an esmp2_status and leaves a
 *    message for esmp2_last_error().
 *  - Orbital order: No occupied then Nv virtual orbitals; virtual a is orbital No+a.
 *  - Two-electron integrals are real chemist-notation (pq|rs) with 8-fold symmetry.
 *  - All arrays are row-major float64 unless stated otherwise.
 *  - The iterative vector ("block vector") is five full-storage blocks
 *    [5][No][No][Nv][Nv] (T, S, X, Y, Z) in the TOP basis; the element meaning,
 *    masks and inner-product weights are returned by esmp2_layout().  Block k
 *    element (i,j,a,b) is the coefficient of the operator string
 *      T: a+_{a up} a+_{b up} a_{j up} a_{i up}|Phi>            (shared with down-down)
 *      S: a+_{a up} a+_{b dn} a_{j dn} a_{i up}|Phi>
 *      X: a+_{t' up} a+_{a up} a+_{b up} a_{j up} a_{i up} a_{t up}|Phi>   (shared, all down)
 *      Y: a+_{t' up} a+_{a dn} a+_{b dn} a_{j dn} a_{i dn} a_{t up}|Phi>   (shared, spin flip)
 *      Z: a+_{a up} a+_{t' dn} a+_{b dn} a_{j dn} a_{t dn} a_{i up}|Phi>   (shared, spin flip)
 *    with t = occupied 0 (largest singular value) and t' = virtual 0 (Eq. psi1).
 *  - Device pointers passed to the library stay owned by the caller; the library
 *    never frees them.  Buffers owned by a handle are released by esmp2_destroy().
 *  - Calls on one handle are not thread-safe; distinct handles are independent.
 */
#ifndef ESMP2_H
#define ESMP2_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  ESMP2_OK = 0,
  ESMP2_ERR_INVALID_ARG = 1,   /* bad size, NULL pointer, non-finite input */
  ESMP2_ERR_UNSUPPORTED = 2,   /* e.g. triplet spin, Nv < No, layout not supported */
  ESMP2_ERR_OOM = 3,           /* device allocation failed */
  ESMP2_ERR_NOT_CONVERGED = 4, /* maxit reached before the residual tolerance */
  ESMP2_ERR_INDEFINITE = 5,    /* CG met p.Ap <= 0: (H0 - E0) is not positive definite */
  ESMP2_ERR_CUDA = 6,          /* a CUDA runtime error (message in esmp2_last_error) */
  ESMP2_ERR_TIMEOUT = 7,       /* a bounded device-side wait gave up */
  ESMP2_ERR_STATE = 8          /* call order violated (e.g. energy before solve) */
} esmp2_status;

typedef enum {
  ESMP2_FP64 = 0,        /* every contraction in float64 */
  ESMP2_MIXED_BF16 = 1,  /* sigma contractions bf16 x bf16 -> fp32 (tcgen05) inside fp64 refinement */
  ESMP2_MIXED_TF32 = 2,  /* as ESMP2_MIXED_BF16 with the inner contraction on float32 operands read as
                            tf32 by the tensor cores (kind::tf32: 10 explicit mantissa bits, low bits
                            of each float32 operand ignored) with fp32 accumulation; the inner PCG
                            vector p is itself the operand.  Packed inner solve only: No <= 32, else
                            ESMP2_ERR_UNSUPPORTED. */
  ESMP2_REDUCED_MIXED = 4, /* the D + L solve in the reduced-cost basis: occupied orbitals other than t
                            and virtual orbitals other than t' diagonalise their blocks of F (D and L
                            are unchanged by rotations that fix t and t', Sec. II.C), so both blocks
                            are a diagonal plus the t / t' row and column and every virtual-index
                            term is element-wise (no N_o^2 N_v^3 contraction).  Float32 inner PCG
                            inside float64 refinement; the right-hand side is rotated once
                            (float64-exact digit-split products).  E2 equals the other forms' to
                            the solve tolerance; E2_S stays in the TOP basis.  No <= 32, Nv <= 1024. */
  ESMP2_REDUCED_MINRES = 5, /* preconditioned MINRES in float64 in the reduced-cost basis (SPD
                            preconditioner |diag|^-1): for operators that are not positive definite
                            (intruder states, strong coupling), where CG stops with INDEFINITE */
  ESMP2_FP64_TC = 3      /* float64-accurate virtual-index terms: x and F_vv split into exact 6-bit
                            bf16 digits (per-slice power-of-two scale), digit products summed exactly
                            in fp32 on tcgen05 level by level (levels 2..10) and combined in float64;
                            other terms float64.  Agrees with float64 GEMMs to a few 1e-15 of each
                            slice's largest element.  Needs Nv < 910 (exact fp32 level sums). */
} esmp2_precision;

typedef struct esmp2_handle esmp2_handle;

/* Problem statement (Sec. II.A, II.C): Fock matrix F built from Psi0's one-body
 * density, the integral blocks the right-hand side Q H Psi0 needs, and C. */
typedef struct {
  int No, Nv;               /* occupied / virtual spatial orbitals; 1 <= No <= 64, No <= Nv */
  const double *F;          /* (No+Nv)^2, symmetric, ESMF orbital basis */
  const double *ovov;       /* (ia|jb)  [No][Nv][No][Nv] */
  const double *ooov;       /* (ij|ka)  [No][No][No][Nv] */
  const double *ovvv;       /* (ia|bc)  [No][Nv][Nv][Nv] */
  const double *C;          /* No x Nv singles coefficients (any normalisation; rescaled so 2|C|^2 = 1) */
  int spin;                 /* +1 singlet (supported); -1 triplet -> ESMP2_ERR_UNSUPPORTED */
  int inputs_on_device;     /* 0: host pointers, 1: device pointers (read during create only) */
  /* Large transition-orbital pairs (Sec. II.C partition of the triples into L / S / N):
   * n_large > 0: the n_large largest singular values; n_large == 0 and eta > 0: every pair with
   * lambda_u > eta; n_large == 0 and eta <= 0: TOP(1), the largest.  This library builds
   * TOP(1): any selection of more than one pair returns ESMP2_ERR_UNSUPPORTED, none
   * ESMP2_ERR_INVALID_ARG. */
  double eta;
  int n_large;
  int avo_convention;       /* completion of the virtual space (AVOs): 0 = Householder QR (only) */
  double level_shift;       /* s added to H0 on the first-order space (A -> A + s, every S-space
                               denominator + s): the intruder-state remedy the paper cites for
                               CASPT2 (Sec. III); 0 = the paper's ESMP2 */
} esmp2_desc;

typedef struct {
  int No, Nv;
  int64_t block_elems;      /* No*No*Nv*Nv */
  int64_t n_elems;          /* 5 * block_elems: length of a block vector */
  double weights[5];        /* determinant inner product = sum_k weights[k] * sum(u_k * v_k) */
  double omega;             /* E0 - E_Phi[F] = sum_u 2 lam_u^2 (F_u'u' - F_uu) */
  double E0;                /* <Psi0|F|Psi0> */
} esmp2_layout_info;

typedef struct {
  int iterations;           /* total CG iterations (inner iterations for mixed precision) */
  int outer;                /* fp64 refinement steps (1 for ESMP2_FP64) */
  int sigma_fp64;           /* number of float64 sigma applications */
  int sigma_lowp;           /* number of low-precision sigma applications */
  double rel_residual;      /* true ||b + A x|| / ||b|| at exit (determinant norm) */
  double seconds;           /* wall time of the solve (host clock) */
} esmp2_solve_info;

typedef struct {
  double E2, E2_D, E2_L, E2_S;   /* E2 = E2_D + E2_L + E2_S (Eh) */
} esmp2_energy_parts;

/* Create a handle: normalises C, builds the TOP basis on the device (one-sided Jacobi
 * SVD of C, Householder completion of the virtual space; Sec. II.A), transforms F and
 * the integrals, builds the right-hand side b = Q H Psi0 on D+L and the diagonal.
 * Inputs are copied; the caller keeps ownership.  Stream: the default stream until
 * esmp2_set_stream().  Errors: INVALID_ARG, UNSUPPORTED, OOM, CUDA. */
esmp2_status esmp2_create(esmp2_handle **h, const esmp2_desc *d);
void esmp2_destroy(esmp2_handle *h);
const char *esmp2_last_error(const esmp2_handle *h);

/* Launch every later kernel of this handle on `stream` (a cudaStream_t, e.g. torch's
 * current stream).  NULL selects the legacy default stream. */
esmp2_status esmp2_set_stream(esmp2_handle *h, void *stream);

esmp2_status esmp2_layout(const esmp2_handle *h, esmp2_layout_info *out);

/* TOP basis as built on the device, copied to host arrays (any may be NULL):
 * U No x No, lam No, Wv Nv x Nv (first No columns = TOP virtuals), F_top (No+Nv)^2. */
esmp2_status esmp2_top_basis(esmp2_handle *h, double *U, double *lam, double *Wv, double *F_top);

/* y = (H0 - E0) x on D+L (the "sigma build"): Eq. qfq_replacement restricted to the
 * doubles and L-triples, minus E0.  x, y: caller-owned DEVICE buffers of n_elems
 * float64 in the block layout; x must be zero on masked elements and antisymmetric
 * where the layout says so; y is written on every element (zero on masked ones).
 * p = ESMP2_FP64 computes in float64; ESMP2_MIXED_BF16 computes it the way the inner solve
 * of the mixed-precision solver does: the N_o^2 N_v^3 virtual-index contractions from bf16
 * operands (fp32 accumulation) as one tensor-core GEMM, everything else in float32, in the
 * basis whose occupied orbitals other than t diagonalise F_oo; for No <= 32 it needs x to
 * have the spin-flip symmetry of the singlet, S_ij^ab = S_ji^ba (every vector of the problem
 * has it: b, the solution and every Krylov vector), and returns y with that symmetry and the
 * antisymmetry of T, X, Y exactly.  ESMP2_MIXED_TF32: the same with the virtual-index
 * contraction on tf32 operands (No <= 32).  ESMP2_REDUCED_MIXED: the inner float32 sigma of the
 * reduced-cost basis (x rotated in, y rotated back; No <= 32).  x and y must not overlap. */
esmp2_status esmp2_sigma(esmp2_handle *h, const double *x, double *y, esmp2_precision p);

/* Per-stage device timing of `reps` sigma builds y = A x (same arguments as esmp2_sigma),
 * measured with CUDA events on the handle's stream; ms[0..7] receives average
 * milliseconds per build.  ESMP2_FP64: [0] virtual-index contractions, [1] occupied-index
 * contractions, [2] coupling intermediates, [3] element-wise coupling pass, [4] total.
 * ESMP2_MIXED_BF16 / ESMP2_MIXED_TF32 (No <= 32, the packed inner sigma on float32 vectors):
 * [0] operand conversion (bf16 rounding; tf32: none, the vector is the operand), [1] transposed Z
 * slices + virtual-index tcgen05 GEMM, [2] 0, [3] arrow sums, intermediates and coupling pass,
 * [4] total.  Not part of the
 * method: it exists so that benchmarks can attribute time to kernels. */
esmp2_status esmp2_profile_sigma(esmp2_handle *h, const double *x, double *y, esmp2_precision p, int reps,
                                 double *ms);

/* The virtual-index contractions alone, y_s = X_s F_vv + F_vv X_s for every slice
 * s = (block, i, j) of the block vector (no masks, couplings or occupied terms):
 * ESMP2_FP64 with float64 GEMMs, ESMP2_MIXED_BF16 with the bf16 tcgen05 kernel (fp32
 * accumulation).  A diagnostic for testing and timing the tensor-core path. */
esmp2_status esmp2_virtual_contraction(esmp2_handle *h, const double *x, double *y, esmp2_precision p);

/* Right-hand side b = Q H Psi0 on D+L (Slater-Condon, Sec. II.B), copied into a
 * caller-owned DEVICE buffer of n_elems float64. */
esmp2_status esmp2_rhs(esmp2_handle *h, double *b);

/* Solve (H0 - E0) x = -b on D+L by Jacobi-preconditioned conjugate gradients
 * (Sec. III.A uses CG).  ESMP2_FP64: plain fp64 PCG.  ESMP2_MIXED_BF16: fp64
 * iterative refinement, each step solving the correction with bf16/fp32 inner
 * PCG.  ESMP2_MIXED_TF32: the same with tf32 inner contractions (No <= 32, else
 * UNSUPPORTED).  ESMP2_REDUCED_MIXED: the same in the reduced-cost basis (see the enum).
 * ESMP2_REDUCED_MINRES: preconditioned MINRES (Paige-Saunders) in float64 in that basis, for
 * operators that are not positive definite; restarted from x until the true residual meets tol.
 * Stops when the TRUE relative residual ||b + A x|| / ||b|| (fp64) <= tol.
 * (Mixed: intermediate true residuals far from tol take fewer exact digit levels and a
 * float32 coupling pass, accurate relative to their own size; the residual that stops
 * the solve, and that the energy reuses, is float64-accurate throughout.)
 * Errors: NOT_CONVERGED (maxit CG iterations in total), INDEFINITE, CUDA.
 * The solution stays on the device (esmp2_get_solution); a later solve warm-starts
 * from it. */
esmp2_status esmp2_solve(esmp2_handle *h, double tol, int maxit, esmp2_precision p, esmp2_solve_info *info);

/* Copy the current solution x (DEVICE buffer, n_elems float64) out / set a guess in. */
esmp2_status esmp2_get_solution(esmp2_handle *h, double *x);
esmp2_status esmp2_set_solution(esmp2_handle *h, const double *x);

/* E2 = E2_D + E2_L + E2_S.  E2_D, E2_L: Hylleraas functional 2 b.x + x.Ax of the
 * current solution (error quadratic in the residual); E2_S = -sum_S b_I^2 / D_I over
 * the S-triples with the diagonal Fock denominator (Sec. II.D), evaluated on the fly.
 * All reductions in float64.  Requires a previous esmp2_solve (else ERR_STATE). */
esmp2_status esmp2_energy(esmp2_handle *h, esmp2_energy_parts *parts);

/* Batched solve of independent instances of uneven No/Nv (e.g. several excited states
 * or molecules).  Each instance i is created from descs[i], solved to the true relative
 * residual tol with precision p, its energy evaluated, and destroyed; results[i] receives
 * the status, energies, solve info and launches of instance i.  `concurrency` host
 * workers each drive their own non-blocking CUDA stream on the current device and take
 * instances in order from a shared counter, so small instances overlap; device memory in
 * use is that of `concurrency` instances at a time.  In the mixed solve of an instance of
 * at most 64M amplitudes the inner PCG iteration is captured once and replayed as a CUDA
 * graph.  p: ESMP2_FP64, ESMP2_FP64_TC, ESMP2_MIXED_BF16, ESMP2_MIXED_TF32 or ESMP2_REDUCED_MIXED.
 * Returns ESMP2_OK if every
 * instance succeeded, else the first failing status (every instance is still attempted). */
typedef struct {
  esmp2_status status;
  esmp2_energy_parts e2;
  esmp2_solve_info info;
  int64_t kernel_launches;
  char message[160];
} esmp2_batch_result;
esmp2_status esmp2_batch_solve(const esmp2_desc *descs, int count, double tol, int maxit, esmp2_precision p,
                               int concurrency, esmp2_batch_result *results);

/* Analytic gradient of E2 (after esmp2_solve, else ESMP2_ERR_STATE) with respect to the
 * inputs F and (ia|jb), in the ESMF orbital basis, written to HOST arrays (either may be NULL):
 *   dF[p][q]           = dE2/dF_pq with E2 evaluated on (F + F^T)/2 (dF is symmetric; a step
 *                        that moves F_pq and F_qp together changes E2 by (dF_pq + dF_qp) h),
 *   dOVOV[i][a][j][b]  = dE2/d(ia|jb) with E2 evaluated on the (ia)<->(jb) symmetrised block.
 * Uses dE2 = 2 <x, db> + <x, dA x> + dE2_S (first-order equation A x = -b, A symmetric, so
 * the adjoint vector is x; the TOP rotation depends on C only).  adjoint_solve != 0 also
 * solves A^T lambda = -b in float64 from zero and returns |lambda - x| / |x| in
 * *adjoint_rel_diff (may be NULL).  The solution in the handle is left unchanged. */
esmp2_status esmp2_grad(esmp2_handle *h, double *dF, double *dOVOV, int adjoint_solve, double *adjoint_rel_diff);

/* Number of CUDA kernels this handle has launched since creation (for accounting). */
int64_t esmp2_kernel_launches(const esmp2_handle *h);

/* Process-wide timing of the kernel families of the hot path (measurement support; the
 * paper has no counterpart).  While enabled, each launch of an instrumented family is
 * bracketed by two CUDA events on the stream it runs on, and its work is recorded:
 *   ESMP2_KT_CONTRACTION  tcgen05 virtual-index contraction with bf16 operands (inner sigma);
 *                         alg_units = the method's flops, 4 n_unique Nv per sigma build
 *                         (n_unique = unique D+L amplitudes, spin-flip pairs once),
 *                         exec_units = flops the tensor cores execute on the stored slices
 *   ESMP2_KT_COUPLING     element-wise coupling pass (five block launches); units = bytes of
 *                         one read of x and one read and write of y
 *   ESMP2_KT_GEMM64       float64 GEMM (transforms, float64 sigma); units = flops
 *   ESMP2_KT_E2S          S-space energy sum; units = S-space elements
 *   ESMP2_KT_DIGITS       float64-accurate contraction from exact bf16 digit products (true
 *                         residual, energy, integral rotations); alg_units = the method's
 *                         flops of ONE contraction (4 n_unique Nv, or 2 rows Nv^2 for a
 *                         rotation), however many digit pairs emulate it; exec_units = the
 *                         tensor-core flops of every digit pair
 *   ESMP2_KT_PRECOND      tcgen05 GEMMs of the inner preconditioner (the two-sided rotation of
 *                         the residual to and from the basis that diagonalises F_vv); units =
 *                         executed flops (extra work, not part of the method's count)
 * esmp2_kernel_times synchronises the recorded events, fills out[ESMP2_KT_COUNT] with the
 * totals since the last call and clears them ("launches" counts timed scopes: one coupling
 * pass, one E2_S sector).  Enabling adds two event records per scope. */
typedef enum {
  ESMP2_KT_CONTRACTION = 0,
  ESMP2_KT_COUPLING = 1,
  ESMP2_KT_GEMM64 = 2,
  ESMP2_KT_E2S = 3,
  ESMP2_KT_DIGITS = 4,
  ESMP2_KT_PRECOND = 5,
  ESMP2_KT_COUNT = 6
} esmp2_kernel_family;
typedef struct {
  int64_t launches;
  double ms;          /* summed event-to-event device time */
  double alg_units;
  double exec_units;
} esmp2_kernel_time;
void esmp2_kernel_timing(int enable);
esmp2_status esmp2_kernel_times(esmp2_kernel_time *out);

/* Allocation-free bf16 virtual-index contraction (the paper has no counterpart; this is a
 * library service).  Computes, like esmp2_virtual_contraction(..., ESMP2_MIXED_BF16),
 *     y_s = X_s F + F X_s   for s = 0..S-1,  X_s = x[s] (Nv x Nv),  F = Fvv (Nv x Nv)
 * with bf16 operands and fp32 accumulation, written to y as float64.  x, Fvv, y are
 * caller-owned DEVICE buffers (S*Nv*Nv, Nv*Nv, S*Nv*Nv float64), on the current device;
 * no handle is needed.
 * For callers that cannot allocate device memory where they call it: code running while
 * another framework owns the whole device heap through its own caching allocator, and
 * latency-critical loops where a cudaMalloc/cudaFree pair would synchronise the device.
 * It calls no cudaMalloc, cudaFree or allocating library routine: its scratch (bf16 copies
 * of x and F, the fp32 accumulator, an error flag) is one file-scope device array of
 * ESMP2_NOALLOC_MAX_BYTES that every GPU loading this library holds until process exit.
 * The scratch needed is 256 + (2 Nv Nvp) + (2 S Nv Nvp) + (4 S Nv Nv) bytes (each term
 * rounded up to 256, Nvp = Nv rounded up to 8); larger requests return
 * ESMP2_ERR_UNSUPPORTED without touching the device.
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress)
 * and caches it.  All calls share the
 * array and it keeps the last call's contents (the error flag is cleared on entry), so
 * calls that overlap on the GPU (different streams or threads) race; serialise them.
 * The call synchronises `stream` (a cudaStream_t, NULL = legacy default) to read the
 * kernel's error flag: ESMP2_ERR_TIMEOUT if a bounded device wait gave up, ESMP2_ERR_CUDA
 * on a CUDA error, ESMP2_ERR_INVALID_ARG on NULL pointers or non-positive sizes. */
#define ESMP2_NOALLOC_MAX_BYTES (64u << 20)
esmp2_status esmp2_virtual_contraction_noalloc(const double *x, const double *Fvv, double *y, int S, int Nv,
                                               void *stream);

/* Self-test of the failure detection of the tensor-core kernel (the paper has no
 * counterpart).  Every mbarrier wait of that kernel is bounded; a wait that runs out raises a
 * device error flag that the host turns into ESMP2_ERR_TIMEOUT, and the CUDA context stays
 * usable.  This call runs one CTA of the kernel on a 16 x 16 dummy slice whose producer issues
 * no copies, so the consumer's first waits run out after wait_ms milliseconds (1 .. 2000) with
 * no copy, MMA or TMEM load in flight.  It returns ESMP2_ERR_TIMEOUT when the expiry was
 * detected and reported (the expected outcome), ESMP2_OK if it was not, ESMP2_ERR_CUDA on a
 * CUDA error, ESMP2_ERR_INVALID_ARG for wait_ms out of range.  It allocates nothing: it uses
 * the scratch array of esmp2_virtual_contraction_noalloc (so it must not overlap such a call
 * on the GPU) and synchronises `stream` (a cudaStream_t, NULL = legacy default). */
esmp2_status esmp2_selftest_bounded_wait(int wait_ms, void *stream);

#ifdef __cplusplus
}
#endif
#endif
