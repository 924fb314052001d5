// Internal structures and kernel launchers of libdpar2.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <string>
#include <vector>

#include "dpar2.h"

namespace dp2 {
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};
}  // namespace dp2

struct dpar2_ctx {
  int device = 0;
  int num_sms = 0;
  std::string err;
  int* d_status = nullptr;  // device status word (dp2::ST_*)
  int* h_status = nullptr;  // pinned mirror (64 bytes: the status word, then scalars read back at byte 8)
  std::map<std::string, dp2::DevBuf> ws;  // named scratch buffers, grow-only
  // learned-sketch forward state kept for the backward pass
  int sk_K = 0, sk_J = 0, sk_ell = 0, sk_LP = 0;
  int64_t sk_N = 0, sk_ldx = 0, sk_maxI = 0;
  const void* sk_X = nullptr;
  dpar2_dtype sk_dtype = DPAR2_F32;
  bool sk_ready = false;
  bool sk_tc = false;                 // 16-bit X on the tensor-core passes
  std::vector<int64_t> sk_toff;       // K + 1 prefix sums of 128-row tiles per slice
  std::vector<int64_t> sk_off2;       // row ranges of the gradient's last pass (64-row aligned)
  std::vector<int64_t> sk_poff2;      // the same, last entry padded to a multiple of 64
  std::vector<int64_t> sk_poff;       // K + 1 offsets of the slices padded to 64 rows (Q split)
  // phase timing (DPAR2_PH_*): start/end events on the work stream
  bool timing = false;
  cudaEvent_t tev[2 * DPAR2_NUM_PHASES] = {};
  bool tpending[DPAR2_NUM_PHASES] = {};
  double tms[DPAR2_NUM_PHASES] = {};
  // scratch buffer of at least `bytes` bytes under `name` (contents undefined);
  // nullptr when the allocation failed
  void* get(const std::string& name, size_t bytes);
  // stream-ordered pool of the compression objects' buffers (memory kept for
  // reuse); the context outlives its last compression object
  cudaMemPool_t pool = nullptr;
  int live_comps = 0;
  bool closing = false;
  // autotuned choices (projection schedule) per problem shape
  std::map<std::string, int> tuned;
  std::string pj_lists_key;  // problem shape whose projection work lists are on the device
  int pj_last_schedule = -1, pj_last_cols = 0;  // the last compression's projection (schedule, width)
  // pinned host staging for the small index tables a call copies to the device
  // (asynchronous copies; a call's regions are reused by the next call, after
  // the synchronisation every call ends with)
  int64_t* hstage = nullptr;
  size_t hstage_cap = 0, hstage_used = 0;
};

struct dpar2_comp {
  dpar2_ctx* owner = nullptr;  // context whose pool and work stream hold the buffers
  int K = 0, J = 0, R = 0, ell = 0, LP = 0;
  int Jq = 0;  // J rounded up to 64: columns of the BF16 parts of M^T held in M
  int64_t N = 0, maxI = 0;
  std::vector<int64_t> h_offsets;
  dp2::DevBuf offsets, A, Bk, M, D, E, Ft, xnorm2, rank1, DtD;
  size_t device_bytes() const;
  ~dpar2_comp();
};

namespace dp2 {

// ---- RNG / operand preparation ----
void launch_gaussian(uint64_t seed, uint32_t stream_id, int64_t n, float* out, int round16, cudaStream_t s);
void launch_philox_words(uint64_t seed, uint32_t stream_id, int64_t n, uint32_t* out, cudaStream_t s);
void launch_pad_omega(const float* om, int J, int ell, int Jpad, int LP, dpar2_dtype dt, float* out,
                      cudaStream_t s);
// packed rows (J elements of es bytes) -> rows of pitch ldx elements, pad columns zeroed
void launch_repitch(const void* src, int64_t rows, int J, int es, void* dst, int64_t ldx, cudaStream_t s);

// ---- stage 1, CUDA-core path ----
void launch_sketch_generic(const void* X, dpar2_dtype dt, int64_t ldx, int64_t N, int J, const float* om_pad,
                           int LP, float* Y, cudaStream_t s);
void launch_sketch_generic_per_slice(const void* X, dpar2_dtype dt, int64_t ldx, const int64_t* d_off, int K,
                                     int maxI, int J, const float* om_k, int Jpad, int LP, float* Y,
                                     cudaStream_t s);
void launch_project_generic(const void* X, dpar2_dtype dt, int64_t ldx, const int64_t* d_off, int K, int J,
                            int Jp, const float* Q, int LP, float* B1, double* xpart, int* nJb_out,
                            cudaStream_t s);
int project_blocks(int Jp, int LP);

// ---- stage 1, tensor-core path (16-bit X, tcgen05 + TMA) ----
bool tc_available();
constexpr int kProjNormWarps = 8;  // partial ||X_k||^2 per column block of the tensor-core projection
int tc_lpn(int ell);  // MMA N width of the sketch: 32 or 64
void launch_omega_t16(const float* om_pad, int Jpad, int LP, int LPN, dpar2_dtype dt, void* out, cudaStream_t s);
bool launch_sketch_tc(const void* X, dpar2_dtype dt, int64_t ldx, int64_t N, int J, const void* omT16, int Jpad,
                      int LPN, int LP, float* Y, int num_sms, int* status, cudaStream_t s);
// Right operand of the tensor-core projection for sketch width l: MMA N (NS:
// 48, 64, 96 or 192) and the row offset OFF between the three 16-bit parts
// (part t of column c in row t OFF + c).
void proj_layout(int ell, int* NS, int* OFF);
// Q rows -> three 16-bit parts per slice in that layout, scaled by a power of
// two that launch_project_tc divides out when called with qscale
void launch_qsplit(const float* Q, int LP, int NS, int OFF, const int64_t* d_off, const int64_t* d_poff, int K,
                   int64_t Npad, int64_t maxPad, dpar2_dtype dt, void* out, cudaStream_t s);
// Work-item width of the tensor-core projection in halves of 128 columns:
// the default (as many as TMEM holds double-buffered) and the narrower
// candidate the autotuner also times (0: none)
int project_hv_default(int NS);
int project_hv_alt(int NS);
// X columns per work item of the tensor-core projection (nJb = ceil(Jp / cols));
// hv 0 = the default width
int project_tc_cols(int NS, int hv = 0);
// false if no tensor map could be made or hv is not a width of this NS
bool launch_project_tc(const void* X, dpar2_dtype dt, int64_t ldx, int64_t N, const int64_t* d_off,
                       const int64_t* d_poff, int K, int J, int Jp, const void* Qs, int64_t Npad, int NS, int OFF,
                       int LP, float* B1, double* xpart, int nJb, bool qscale, int num_sms, int* status,
                       cudaStream_t s, const int* lptr = nullptr, const int* items = nullptr, int nlists = 0,
                       int hv = 0);
// Work lists of the tensor-core projection (items k nJb + jb): longest slices
// first, each onto the least-loaded of `nlists` CTAs.  Host side; lptr gets
// nlists + 1 entries, items K nJb.
void project_lpt_lists(const int64_t* row_offsets, int K, int nJb, int nlists, std::vector<int>& lptr,
                       std::vector<int>& items);

// per-slice right operand (three 16-bit parts, [k][3 LPN][Jpad]); ntiles = sum_k ceil(I_k / 128)
bool launch_sketch_seg_tc(const void* X, dpar2_dtype dt, int64_t ldx, int64_t N, int J, const int64_t* d_off,
                          const int64_t* d_toff, int64_t ntiles, int K, const void* Ms, int Jpad, int LPN, int LP,
                          float* U, int num_sms, int* status, cudaStream_t s);

// ---- learned sketch (range-finder loss and its gradient) ----
// per slice: ratio_k, P_k, S_k (K x LP x LP); out = mean ratio
void launch_sl_loss(const float* M1, const float* M2, const double* GB, const double* xn, int K, int ell, int LP,
                    double* ratio, float* P, float* S, double* out, cudaStream_t s);
// rows of B1 as the per-slice right operand of X_k B1_k^T (16-bit parts [k][3 LPN][Jpad]
// or FP32 [k][Jpad][LP]), each row times a power of two (rscale: K x LP)
void launch_sl_rowsplit(const float* B1, int K, int Jp, int J, int Jpad, int ell, int LP, int LPN, dpar2_dtype dt,
                        void* out16, float* out32, float* rscale, cudaStream_t s);
// W rows (FP32, N x LP) and the largest |W| per column (wmax[LP]); bmax: scratch of
// sl_wrows_blocks(K, maxI) x LP floats
int64_t sl_wrows_blocks(int K, int64_t maxI);
void launch_sl_wrows(const float* U, const float* Q1, const int64_t* d_off, int K, int64_t maxI, int LP,
                     const float* P, const float* S, const double* xn, double gscale, const float* rs, float* W,
                     float* bmax, unsigned* wmax, cudaStream_t s);
void launch_sl_wsplit(const float* W, int64_t N, int LP, int LPN, const unsigned* wmax, dpar2_dtype dt, void* out16,
                      cudaStream_t s);
void launch_sl_gradsum(const float* part, int np, int LP, int Jp, int J, int ell, const unsigned* wmax, float* grad,
                       cudaStream_t s);

// ---- per-slice small linear algebra ----
// G[k] = Y_k^T Y_k (FP64, pitch LP).  nsplit > 1 splits every slice's rows over
// nsplit blocks (partials in Gpart, K * nsplit * LP * LP) for few long slices.
// Double-float accumulation of exact products (both CholeskyQR steps).
void launch_gram_dd(const float* Y, int LP, const int64_t* d_off, int K, int ell, double* G, double* Gpart,
                    int nsplit, cudaStream_t s);
// fp64: factorise in FP64 (first CholeskyQR step) or FP32 (second step).
void launch_chol_drop(const double* G, int K, int ell, int LP, double tau, float* Minv, int* rank, int* status,
                      bool fp64, cudaStream_t s);
// Y <- Y Minv_k per slice (Q1 of the first CholeskyQR step) and G = the Gram
// of the new Y, in one pass (partials and their sum as launch_gram_dd)
void launch_formq_gram(float* Y, int LP, const int64_t* d_off, int K, int ell, const float* Minv, double* G,
                       double* Gpart, int nsplit, cudaStream_t s);
void launch_reduce_rows_f64(const double* part, int K, int n, double* out, cudaStream_t s);
void launch_gram_b1(const float* B1, int Jp, int J, int K, int ell, int LP, double* G, cudaStream_t s);
void launch_eig_top(const double* G, const float* M2, int K, int ell, int LP, int R, float* T, float* lam,
                    int* status, cudaStream_t s);
// register-resident variant (one-sided Jacobi on the Cholesky factor); false for LP > 32
bool launch_eig_wide(const double* G, const float* M2, int K, int ell, int LP, int R, float* T, float* lam,
                     int* status, cudaStream_t s);
bool launch_eig_reg(const double* G, const float* M2, int K, int ell, int LP, int R, float* T, float* lam,
                    int* status, cudaStream_t s);
// M_k blocks written as M^T (rows k R + r, Jq columns) in three BF16 parts,
// part p at Ms + p pstride elements (Ms: the first row of the K slices given)
void launch_mblock(const float* B1, int Jp, int J, int K, int ell, int LP, int R, float* T, float* Bk, void* Ms,
                   int64_t pstride, int Jq, int* rank, float tau, cudaStream_t s);
void launch_seg_product(const float* In, int ldin, int nin, const float* T, int64_t tstride, int nout, float* Out,
                        int ldout, const int64_t* d_off, int K, int64_t maxI, cudaStream_t s);

// ---- stage 2 ----
// Tensor-core passes over the BF16 parts of M^T (Ms: 3 x KR x Jq): the sketch
// (part[c] = J x LP partial of M Omega2) or the projection (part[c] = KR x LP
// partial of M^T Q2); Bs = the right operand split by launch_s2_split_rhs
// (s2_nb(LP) x bcols, bcols = KR rounded up to 64 for the sketch, Jq for the
// projection); nch chunks from s2_tc_chunks.  False if no tensor map could be
// made.
int s2_nb(int LP);
int s2_tc_chunks(bool sketch, int64_t KR, int J, int Jq, int num_sms);
bool launch_s2_tc(bool sketch, const void* Ms, int64_t KR, int J, int Jq, const void* Bs, int64_t bcols, int LP,
                  float* part, int nch, int num_sms, int* status, cudaStream_t s);
void launch_s2_split_rhs(const float* F, int64_t nf, int LP, int64_t bcols, void* Bs, cudaStream_t s);
// M (K x J x R FP32) from the parts (inspection)
void launch_ms_to_m(const void* Ms, int64_t pstride, int K, int J, int Jq, int R, float* M, cudaStream_t s);
void launch_sum_parts(const float* part, int nparts, int64_t n, float* out, cudaStream_t s);
// E_r = ||Ft(:, r)||, dropped columns zeroed in Ft and D.  part: kEnormBlocks x R
// doubles, keep: R floats, ndrop: 1 int (device scratch).
constexpr int kEnormBlocks = 304;
void launch_s2_enorm(float* Ft, int64_t rows, int R, float* D, int J, float* E, float tau, double* part,
                     float* keep, int* ndrop, cudaStream_t s);
// out (n x n, FP64) = A^T B over `rows` rows: block partials over row chunks
// (part: kAtbBlocks x n x n floats of scratch), summed in a fixed order.
constexpr int kAtbBlocks = 64;
void launch_atb(int64_t rows, int n, const float* A, const float* B, double* out, float* part, cudaStream_t s);

// ---- ALS (Alg. 3 repeat loop) ----
// Work of pre_solve (small_solve.cuh): Inv = (A o B)^+ with A = W^T W, reduced
// first from the W-update partials part3 when part3 is non-null and it > 0.
struct PreSolve {
  int R = 0;
  const float* part3 = nullptr;
  int nparts = 0, pstride = 0, it = 0;
  double* WtW = nullptr;
  const double* B = nullptr;
  double* loss = nullptr;
  double* Inv = nullptr;
  double* L = nullptr;  // R x R work arrays of the pseudoinverse fallback
  double* V = nullptr;
  int* status = nullptr;
};

struct AlsBufs {
  int K, J, R;
  const float* D;     // J x R
  const float* Ft;    // K x R x R  (F^(k) E)
  const double* DtD;  // R x R
  float* H;           // R x R
  float* W;           // K x R
  float* CV;          // R x R, V = D CV after the first iteration
  float* Upol;        // K x R x R
  float* Pi;          // K x R x R  (P_k Z_k^T F^(k) E)
  float* Prot = nullptr;  // K x R x R right rotations P_k of the last Q-step (warm start), or null
  const int* rank = nullptr;  // K stage-1 ranks (bound the rank of T_k in the Q-step), or null
  double* Psi;        // R x R  D^T V
  double* VtV;        // R x R
  double* HtH;        // R x R
  double* WtW;        // R x R
  double* Ginv;       // R x R  (V^T V * H^T H)^+
  double* InvH = nullptr;  // R x R  (W^T W * V^T V)^+ from the Q-step's extra block, or null
  double* InvV = nullptr;  // R x R  (W^T W * H^T H)^+ from the Lemma 2 grid's extra block, or null
  float* part;        // 3 regions x pr x (2 R^2 + 2) block partials
  double* loss;       // max_iter history (device)
  double* small;      // scratch, 8 R^2 + 8 doubles
  float* atb;         // scratch of launch_atb, kAtbBlocks R^2 floats
  int* status;
  int nblk;      // blocks of the Lemma 2 / 3 kernels (partials in regions 2, 3)
  int nq = 0;    // blocks of the Q-step (Lemma 1 partials in region 1)
  int pr = 0;    // partials per region of `part` (max(nblk, nq))
  int pstride = 0;  // floats per partial when not 2 R^2 + 2
};
// Persistent ALS kernel (k_als_persist.cu): every iteration of a fit in one
// cooperative launch of one block per SM, for R <= 20.
struct PersistArgs {
  int K, R, max_iter;
  int pstride;  // floats per partial (2 R^2 + 2 rounded up to a multiple of 4)
  int wstride;  // per-warp shared scratch (set by the launcher)
  const float* Ft;
  const double* DtD;
  const int* rank;
  float *H, *W, *CV, *Upol, *Pi, *Prot;
  double *Psi, *VtV, *HtH, *WtW, *Ginv, *InvH, *InvV;
  float *part1, *part2, *part3;  // num_sms - 1 partials each
  double* loss;
  int* status;
  unsigned* bar;  // 3 words of device scratch (zeroed by the launcher)
  int* abort;     // set by the launcher (bar + 2)
};
bool persist_supported(int R);
int64_t persist_capacity(int R, int num_sms);
// Post-fit analyses (k_analytics.cu).
// parts: 3 K ldp bf16 values of scratch; nrm: K doubles.
bool launch_similarity(int K, int L, const float* U, int64_t ldu, double gamma, float* S, int64_t lds, void* parts,
                       int ldp, double* nrm, int num_sms, int* status, cudaStream_t s);
void launch_topk(int nrows, int n, const float* sc, int64_t ld, const int* exclude, int k, int* idx, float* val,
                 cudaStream_t s);
int rwr_max_queries();
void launch_rwr(int K, const float* S, int64_t lds, int nq, const int* tgt, double c, int iters, double* deg,
                float* r, float* y0, float* y1, cudaStream_t s);
void launch_feature_pcc(int J, int R, const float* V, float* Vn, float* C, cudaStream_t s);
bool launch_als_persist(PersistArgs& a, int num_sms, cudaStream_t s);
void launch_als_init(AlsBufs& b, const float* V0, cudaStream_t s);
void launch_als_iteration(AlsBufs& b, int it, cudaStream_t s);
void launch_als_finish(AlsBufs& b, int it, cudaStream_t s);
// Three-launch iteration (k_als3.cu) for R <= 32: the H and V updates formed
// in every block of the grids that need them; nblk = als3_blocks(...)
bool als3_supported(int R);
int als3_blocks(int K, int R, int num_sms);
void launch_als_iteration3(AlsBufs& b, int it, cudaStream_t s);
int als_blocks(int K, int R, int num_sms);
void launch_qstep_only(AlsBufs& b, cudaStream_t s);
// register-resident Q-step (R <= 32: lane = column; 32 < R <= 64: the warp-pair
// kernel); false for R > 64.  `pre`: run pre_solve in an extra block
bool launch_qstep_reg(const AlsBufs& b, float* part, int pstride, int want_g1, cudaStream_t s,
                      const PreSolve* pre = nullptr);
bool launch_qstep_wide(const AlsBufs& b, float* part, int pstride, int want_g1, cudaStream_t s,
                       const PreSolve* pre = nullptr);
int qstep_wide_blocks(int K, int R, int cap);
// blocks of the Q-step launch for K slices at rank R (one wave of resident blocks when it fits)
int qstep_blocks(int K, int R, int nblk);
void launch_upol_h(int K, int R, const float* Upol, const float* H, float* Tk, cudaStream_t s);
void launch_p_from_cv(int K, int R, const float* CV, const float* Ft, float* P, cudaStream_t s);
void launch_vtm(int K, int J, int R, const float* V, const void* Ms, int64_t pstride, int Jq, float* P,
                cudaStream_t s);
void launch_psi_vtv(int J, int R, const float* D, const float* V, double* Psi, double* VtV, float* part,
                    cudaStream_t s);
// AtA (K x ldg x ldg FP64, A_k^T A_k) or null for orthonormal A_k
void launch_fitness(int K, int R, const float* P, const float* Upol, const float* H, const float* W,
                    const double* VtV, const double* xnorm2, double* part, int nblk, double* out, cudaStream_t s,
                    const double* AtA = nullptr, int ldg = 0);
// P_k = V^T (A_k^T X_k)^T from the projection rows B (K x LP x Jp)
void launch_p_stream(int K, int J, int Jp, int R, int LP, const float* V, const float* B, float* P, cudaStream_t s);

}  // namespace dp2
