// Internal declarations of the ESMP2 GB300 library (not part of the C ABI).
#pragma once
#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <cstdint>
#include <string>

#include "../../include/esmp2.h"

namespace esmp2 {

constexpr int kBlocks = 5;  // T, S, X, Y, Z
enum Block { BT = 0, BS = 1, BX = 2, BY = 3, BZ = 4 };

// Determinant inner-product weights of the full-storage blocks: T, X, Y hold every
// unique amplitude four times and stand for two determinants (spin flip); S elements
// are unique determinants; Z elements stand for a determinant and its spin flip.
constexpr double kWeights[kBlocks] = {0.5, 1.0, 0.5, 0.5, 2.0};

struct Dims {
  int No, Nv, N;
  int64_t B;   // block elements No*No*Nv*Nv
  int64_t n;   // 5*B
};

// Strided batched float64 GEMM: C[b](m,n) = alpha * sum_k A[b](m,k) B[b](k,n) + beta * C[b](m,n)
// Optional K split (Kin > 0): k = k1 * Kin + k0 is addressed as k1 * sAk1 + k0 * sAk in A and
// k1 * sBk1 + k0 * sBk in B (a sum over slices and one index of each slice in one GEMM).
struct Gemm64 {
  int M, N, K, batch;
  double alpha, beta;
  const double *A; int64_t sAm, sAk, sAb;
  const double *B; int64_t sBk, sBn, sBb;
  double *C; int64_t sCm, sCn, sCb;
  int Kin;
  int64_t sAk1, sBk1;
};
void gemm64(const Gemm64 &g, cudaStream_t st);

// Mode product of a 4-index tensor: out[..k'..] = sum_k in[..k..] R[k][k'] on axis `mode`;
// R is Kin x Kout with row stride ldR.
void mode_product(const double *in, double *out, const int dims[4], int mode, const double *R,
                  int Kout, int64_t ldR, cudaStream_t st);

// Device intermediates of the N^4 coupling terms of sigma (compute type CT).
template <typename CT>
struct CouplingsT {
  CT *VX;  // [No][No][Nv]  sum_c Fov[0][c] X[i][j][c][b]
  CT *OX;  // [No][Nv][Nv]  sum_k Fov[k][0] X[k][j][a][b]
  CT *WZ;  // [No][No][Nv]  sum_c Fov[0][c] Z[i][j][a][c]
  CT *OZ;  // [No][Nv][Nv]  sum_k Fov[k][0] Z[i][k][a][b]
  CT *G;   // [No][Nv]      sum_kc Fov[k][c] (X+Z)[k][j][c][b]
  CT *GP;  // [No][No][Nv]  sum_c Fov[k][c] (X+Z)[k][j][c][b]   (partial of G)
  CT *HP;  // [No][No][Nv]  sum_c Fov[j][c] (Y+Z)[i][j][a][c]   (partial of H)
  CT *H;   // [No][Nv]      sum_kc Fov[k][c] (Y+Z)[i][k][a][c]
  CT *CYZ; // [No][Nv]      sum_d Fvv[0][d] Z[0][k][d][c] - sum_l Foo[l][0] Z[l][k][0][c]
  CT *OC1; // [5][No][Nv][Nv] sum_{l>=1} Foo[l][0] x[blk][l][j][ab]   (arrow form only)
  CT *OC2; // [5][No][Nv][Nv] sum_{l>=1} Foo[l][0] x[blk][i][l][ab]   (arrow form only)
};
using Couplings = CouplingsT<double>;

struct Solver64 {
  double *x, *r, *p, *q, *w;  // fp64 vectors (n)
};

// Packed layout of the inner (float32) solve.  T, X and Y keep the slices i < j only (slice
// (j, i) is the negative of (i, j)); S and Z keep every slice.  Rows are padded to
// Nvp = Nv rounded up to 8 (pad columns zero).  Slice order T | S | X | Y | Z; the bf16
// operand of the contraction appends the transposed Z slices.  Determinant inner-product
// weights per stored element: 1 for T, S, X, Y (an i < j slice stands for itself and its
// negative partner) and 2 for Z.
struct Packed {
  int No, Nv, Nvp, nh, NN;   // nh = No (No - 1) / 2, NN = No^2
  int64_t SL;                // elements per slice, Nv * Nvp
  int64_t boff[6];           // first element of T, S, X, Y, Z and of the transposed-Z part
  int nslices;               // slices of a packed vector, 3 nh + 2 NN
  int64_t n;                 // elements of a packed vector
};
Packed make_packed(int No, int Nv);

}  // namespace esmp2

struct esmp2_handle {
  esmp2::Dims d;
  cudaStream_t stream = nullptr;
  std::string err;
  int64_t launches = 0;
  // TOP basis and transformed one-electron quantities
  double *C = nullptr;      // No x Nv normalised
  double *U = nullptr;      // No x No
  double *lam = nullptr;    // No
  double *Wv = nullptr;     // Nv x Nv
  double *W = nullptr;      // N x N block-diagonal rotation
  double *F = nullptr;      // N x N  F in the TOP basis
  double *f0vo = nullptr;   // Nv x No  Fock matrix of Phi, virtual-occupied block
  double *scal = nullptr;   // device scalars: [0] omega, [1] E0
  double omega = 0, E0 = 0;
  double level_shift = 0;   // added to H0 on the first-order space
  double omega_op = 0;      // omega - level_shift: the constant of the operator A = F_N - omega_op
  double eta = 0;           // large-pair threshold (TOP(1) checks)
  int n_large = 0;
  // transformed integrals
  double *ovov = nullptr;   // (ia|jb)  No Nv No Nv
  double *ooov = nullptr;   // (ij|ka)  No No No Nv
  double *ovvt = nullptr;   // (ia|bu') No Nv Nv No
  // vectors
  double *b = nullptr;      // right-hand side (n)
  esmp2::Solver64 s64{};
  esmp2::Couplings cp{};
  esmp2::CouplingsT<float> cp32{};
  float *F32 = nullptr;     // float copy of Fsemi (inner solve)
  float arrow_w[64] = {};   // host copy of F32[l][0] (1 <= l < No) and F32[l][No] (l < No)
  bool arrow_w_ready = false;
  __half *dinv32 = nullptr; // Jacobi preconditioner in that basis (n halves)
  double *P64 = nullptr;    // x F for the T, S, X, Y blocks (float64 sigma workspace, 4 blocks)
  double *red = nullptr;    // reduction partials
  double *red_out = nullptr;// reduction results (device)
  double *hred = nullptr;   // pinned host copy of reduction results
  bool solved = false;
  bool e2s_done = false;
  double e2s = 0;
  // low-precision sigma workspace (mixed path)
  void *xlp = nullptr;      // bf16 copy of the sigma input (n)
  void *Fvlp = nullptr;     // bf16 Fvv (Nv x Nv, padded)
  float *ylp = nullptr;     // fp32 sigma output (n)
  float *r32 = nullptr, *p32 = nullptr, *q32 = nullptr, *x32 = nullptr;  // inner PCG vectors
  int *dflag = nullptr;     // device error flag of bounded waits (tcgen05 kernel)
  // basis whose occupied orbitals 1..No-1 diagonalise F_oo (mixed-precision solves)
  bool mixed_ready = false;
  double *Rocc = nullptr, *Rocct = nullptr;  // No x No rotation and its transpose
  double *Fsemi = nullptr;  // N x N
  double *bsemi = nullptr;  // right-hand side in that basis (n)
  int x_basis = 0;          // basis of s64.x: 0 TOP, 1 semicanonical-occupied, 2 reduced-cost
  // reduced-cost basis (occupied orbitals other than t and virtual orbitals other than t'
  // diagonalise their blocks; F is "arrow" shaped in both): ESMP2_REDUCED_MIXED
  bool arrow_ready = false;
  bool arrowv = false;      // the current call works in the reduced-cost basis
  double *Rv = nullptr, *Rvt = nullptr;  // Nv x Nv virtual rotation (t' fixed) and its transpose
  int vrot_level = 0;       // 0 none, 1 to 1e-2 (preconditioner), 2 to the rounding level
  double *jB = nullptr, *jJ = nullptr;  // Jacobi state (rotated rows, accumulated rotation)
  unsigned *jflag = nullptr;
  double *mr_a = nullptr, *mr_b = nullptr, *mr_v = nullptr;  // MINRES direction vectors and Lanczos vector (n)
  void *Rvdig = nullptr, *Rvtdig = nullptr;  // their digit planes (float64-exact rotations)
  int eRv = 0, eRvt = 0;
  double *Farr = nullptr;   // N x N Fock matrix in that basis
  double *barr = nullptr;   // right-hand side in that basis (n)
  float *F32arr = nullptr;  // float copy of Farr (inner solve)
  double *rho64 = nullptr, *kap64 = nullptr;  // [5 No^2][Nv] row / column sums against F_t'c
  float *pRho = nullptr, *pKap = nullptr;     // packed inner: [slices][Nv] row sums, [No^2][Nv] Z column sums
  int pdinv_basis = -1;     // basis the packed preconditioner was built for
  // rotated Jacobi preconditioner of the packed bf16 / tf32 inner solve: z = R D^-1 R^T r per
  // slice, R the virtual rotation that diagonalises F_vv, D the diagonal of A in that basis
  bool rj = false;          // in use for the current solve
  bool rj_ready = false;
  void *pRbf = nullptr, *pT1 = nullptr;  // bf16 r and the intermediate products (packed)
  float *pZ = nullptr;      // z = M^-1 r (packed)
  void *pWR = nullptr, *pWRt = nullptr;  // bf16 right operands for X R and X R^T
  float *pLam = nullptr, *pOcc = nullptr;  // diagonal of F_vv in that basis; per-slice occupied part
  int *pCode = nullptr;     // per-slice block | 8 (i == 0) | 16 (j == 0)
  double *pdot2 = nullptr;  // partials of <r, z>_w
  double *zero_slots = nullptr;  // 32 zero doubles (alpha = beta = 0)
  cudaEvent_t ovvv_ready = nullptr;  // create: the OVVV input copy (side stream) has landed
  bool x_zero = true;       // s64.x is known to be zero (its sigma is zero, no build needed)
  bool r_true = false;      // s64.r holds the true residual -b - A x of s64.x (same basis)
  // float64-accurate virtual-index terms from exact bf16 digit products (tcgen05)
  void *xdig = nullptr;     // digit planes of x [levels-1][5 No^2][Nv][Nvp] bf16
  void *Fdig = nullptr;     // digit planes of F_vv [levels-1][Nv][Nvp] bf16
  int *es = nullptr;        // per-slice exponents (5 No^2) and that of F_vv (last entry)
  int *slist = nullptr;     // slices of the symmetric form (T, X, Y with i < j; all S, Z)
  int nslist = 0, eF = 0;
  void *Rdig = nullptr;     // digit planes of W_v^T (integral transforms on the tensor cores)
  int eR = 0;
  int last_precision = 0;   // precision of the last solve (the energy's sigma follows it)
  cudaGraphExec_t inner_graph = nullptr;  // one inner PCG iteration of the mixed solve
  int64_t inner_graph_launches = 0, inner_graph_launches_pending = 0;
  // packed inner solve (No <= 32): layout, vectors, operand, products and intermediates
  bool packed = false;
  esmp2::Packed pk{};
  float *pr = nullptr, *pp = nullptr, *pq = nullptr, *pd = nullptr;  // r, p, q = A p, correction d
  __half *pdinv = nullptr;  // Jacobi preconditioner (packed)
  void *pop = nullptr;      // bf16 operand: packed p and the transposed Z slices
  void *pW = nullptr;       // bf16 right operand F_vv
  // ESMP2_MIXED_TF32: the operand is float32 read as tf32 by the tensor cores, and the inner
  // PCG's p lives in its first n elements (no separate operand copy)
  bool tf32 = false;        // inner operand kind of the current call
  int graph_kind = -1;      // inner sigma kind (tf32 + 2 reduced basis) the captured iteration was built with
  float *pop32 = nullptr;   // float32 operand: packed p, then the transposed Z slices
  float *pW32 = nullptr;    // float32 right operand F_vv
  float *pP = nullptr;      // products: P (T .. Z slices, row pitch Nvp) then F Z (transposed part)
  float *pVX = nullptr, *pGP = nullptr, *pWZ = nullptr, *pHP = nullptr;  // [No][No][Nv] coupling sums
  float *pOC = nullptr;     // [5][No][SL] arrow sums over the first occupied index (OC1)
  float *pOC2 = nullptr;    // [2][No][SL] arrow sums over the second index (S, Z)
  float *pOX = nullptr, *pOZ = nullptr;  // [No][SL] sum_l F_l,t' X_lm, sum_m F_m,t' Z_lm
  float *pG = nullptr, *pH = nullptr, *pCYZ = nullptr;  // [No][Nv]
  double *pdot = nullptr;   // per-CTA partials of the coupling pass's <p, A p>
  int pdot_n = 0;
};

namespace esmp2 {
// kernels.cu
esmp2_status setup_top_basis(esmp2_handle *h);
esmp2_status setup_rhs(esmp2_handle *h);
esmp2_status sigma64(esmp2_handle *h, const double *x, double *y, int tc_levels = 0);
// s_sym: x has the spin-flip symmetry of S exactly (S_ij^ab = S_ji^ba bit for bit); the
// digit-level virtual pass then contracts the S slices with F_vv from one side only
esmp2_status sigma64_F(esmp2_handle *h, const double *F, int arrow, const double *x, double *y, int tc_levels = 0,
                       int couplings = 1, bool s_sym = false);
void couple_f32_into(esmp2_handle *h, const double *x, double *y);
void launch_intermediates64(esmp2_handle *h, const double *F, int arrow, const double *x);
void launch_couple64(esmp2_handle *h, const double *F, int arrow, const double *x, double *y);
esmp2_status sigma64_tail(esmp2_handle *h, const double *F, int arrow, const double *x, double *y);
esmp2_status virtual_contraction(esmp2_handle *h, const double *x, double *y, int mode);
void contractions64(esmp2_handle *h, const double *F, const double *x, double *y, int stage);
// dot (optional, couple_dot_parts(h) doubles): per-CTA partials of the weighted <x, y>
void couple32(esmp2_handle *h, const float *F32, const float *x, float *y, double *dot = nullptr);
int64_t couple_dot_parts(const esmp2_handle *h);
esmp2_status sigma_mixed(esmp2_handle *h, const double *x, double *y);
esmp2_status profile64(esmp2_handle *h, const double *x, double *y, int reps, double *ms, int tc_levels = 0);
esmp2_status profile_mixed(esmp2_handle *h, const double *x, double *y, int reps, double *ms);
esmp2_status solve64(esmp2_handle *h, double tol, int maxit, esmp2_solve_info *info, int virt_tc = 0);
esmp2_status solve_minres(esmp2_handle *h, double tol, int maxit, esmp2_solve_info *info);
esmp2_status solve_mixed(esmp2_handle *h, double tol, int maxit, esmp2_solve_info *info, bool tf32 = false,
                         bool arrowv = false);
esmp2_status energy(esmp2_handle *h, esmp2_energy_parts *parts);
esmp2_status gradient(esmp2_handle *h, double *dF, double *dOVOV, int adjoint, double *adj_diff);
esmp2_status check_cuda(esmp2_handle *h, cudaError_t e, const char *what);
esmp2_status ensure_mixed(esmp2_handle *h, bool semi);
esmp2_status sigma_inner(esmp2_handle *h, const float *p, float *q, bool p_bf16_ready = false, double *dot = nullptr);
esmp2_status check_device_flag(esmp2_handle *h);
// packed inner solve (inner.cu)
esmp2_status packed_setup(esmp2_handle *h);
esmp2_status sigma_packed(esmp2_handle *h, const float *p, float *q, bool pb_ready, double *dot, int stages = 7);
esmp2_status profile_packed(esmp2_handle *h, const double *x, int reps, double *ms);
void packed_init(esmp2_handle *h, const double *r64, int grid);
esmp2_status packed_rj_setup(esmp2_handle *h);
void k_finalize_ext(const double *red, int nparts, double *slots, int mode, cudaStream_t st);
esmp2_status packed_rj_init(esmp2_handle *h, const double *r64, int grid);
esmp2_status packed_rj_step(esmp2_handle *h, int grid);
esmp2_status ensure_vrot(esmp2_handle *h, bool exact);
float *packed_p(esmp2_handle *h);
void packed_accumulate(esmp2_handle *h, double *x64);
double packed_wdot(esmp2_handle *h, const float *u, const float *v);
esmp2_status sigma_mixed_packed(esmp2_handle *h, const double *x, double *y);
void antisym_project(esmp2_handle *h, double *v);
void singlet_project(esmp2_handle *h, double *v);
void combine_sym(esmp2_handle *h, double *y);
void combine_s(esmp2_handle *h, double *y);
constexpr int kFp64TcLevels = 10;  // digit levels of the float64-exact tensor-core contraction
int split_levels_for(double tol);
bool split_supported(const esmp2_handle *h, int levels);
esmp2_status ensure_split(esmp2_handle *h);
esmp2_status ensure_slist(esmp2_handle *h);
esmp2_status virt_split(esmp2_handle *h, const double *x, double *y, double *p64, int sym, int levels);
esmp2_status xwv_split(esmp2_handle *h, const double *X, int64_t rows, double *Y);
esmp2_status xwm_split(esmp2_handle *h, const double *X, int64_t rows, double *Y, const double *M, void **dig,
                       int *eM, int eslot);
// reduced-cost basis (arrowv.cu)
esmp2_status ensure_arrow(esmp2_handle *h);
esmp2_status rotate_virt(esmp2_handle *h, const double *in, double *out, double *tmp, bool to_arrow);
esmp2_status x_to_basis(esmp2_handle *h, int target);
esmp2_status sigma64_arrow(esmp2_handle *h, const double *x, double *y, int couplings = 1);
void virt_arrow64(esmp2_handle *h, const double *x, double *y);
void rotate_occ(esmp2_handle *h, const double *in, double *out, double *tmp, bool to_semi);
void mode_product_small(const double *in, double *out, int64_t P, int K, int64_t Q, const double *R,
                        cudaStream_t st);
void eigvecs_block(esmp2_handle *h, const double *F, int off, int m, double *V, double *work);
inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Device memory owned by handles: stream-ordered allocations from the device's default
// memory pool, which keeps up to a third of the device memory cached after frees, so a
// handle created after another one reuses its memory without a synchronising
// cudaMalloc/cudaFree pair.  dfree releases in stream order (after the stream's work).
cudaError_t dmalloc(void **p, size_t bytes, cudaStream_t st);
void dfree(void *p, cudaStream_t st);

// Raise the dynamic shared-memory limit of kernel `func` to `bytes` on the current device,
// once per (device, kernel) for the life of the process (the attribute is per device, and
// concurrent callers such as batch workers must not race on it).  Returns the status of
// that one cudaFuncSetAttribute call.
cudaError_t smem_limit_once(const void *func, int bytes);

// 2-D tensor map of bf16 (f32 = false) or float32 elements (inner dimension first; rows of
// row_bytes), box box_inner x box_outer, shared-memory swizzle of 128, 64, 32 or 0 bytes, zero
// fill out of bounds.  False when the CUDA driver's tensor-map encoder is unavailable or
// rejects the description.
bool tma_map_2d(CUtensorMap *m, const void *base, bool f32, uint64_t inner, uint64_t outer, uint64_t row_bytes,
                uint32_t box_inner, uint32_t box_outer, int swizzle_bytes);

// Output options of the virtual-index GEMM (vgemm.cu): transposed rows stored as bf16 into
// PT16 (instead of float32 into PT), optionally scaled by the reduced-cost-basis inverse
// diagonal (lam: [Nv] diagonal of F_vv in that basis, occ: [slices] occupied part, code:
// [slices] block | 8 (i == 0) | 16 (j == 0)); family: kernel-timing family of the launch.
struct VgemmOut {
  void *PT16 = nullptr;
  const float *lam = nullptr, *occ = nullptr;
  const int *code = nullptr;
  int family = 0;
};

// ESMP2_DEBUG=1: synchronise the handle's stream and print the host time since the last
// phase mark (set-up breakdowns; no effect otherwise).
void debug_phase(esmp2_handle *h, const char *name);

// Process-wide kernel timing (esmp2_kernel_timing): a scope records one event pair around
// the launches it encloses when timing is on.
class KScope {
 public:
  KScope(cudaStream_t st, int family, double alg_units, double exec_units);
  ~KScope();
  KScope(const KScope &) = delete;
  KScope &operator=(const KScope &) = delete;
 private:
  cudaStream_t st_;
  int fam_;
  double alg_, exec_;
  cudaEvent_t a_ = nullptr, b_ = nullptr;
};
// unique D+L amplitudes of TOP(1) (spin-flip pairs counted once) and the algorithmic flops
// of the virtual-index terms of one sigma build: 2 flops x 2 virtual sums of length Nv each
double unique_amplitudes(int No, int Nv);
inline double alg_virtual_flops(int No, int Nv) { return 4.0 * unique_amplitudes(No, Nv) * Nv; }
}  // namespace esmp2
