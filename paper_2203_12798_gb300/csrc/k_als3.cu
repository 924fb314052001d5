// ALS iteration in three grid launches (Alg. 3 repeat loop; Lemmas 1-3) for
// ranks R <= 32, whose small solves fit one block's shared memory:
//   1. Q-step grid (k_qstep_reg, unchanged): the Q-steps and the Lemma 1
//      partials; its extra block closes the previous iteration (W^T W and e
//      from the W-update partials) and factors W^T W * V^T V (FP64).
//   2. k_als_hg2: every block reduces the Lemma 1 partials and forms the H
//      update itself (H = G1 (W^T W * V^T V)^-1 in FP64, columns normalised,
//      H rounded to FP32 and H^T H formed from the rounded values), then adds
//      its share of the Lemma 2 partials (double-float); the extra block
//      factors W^T W * H^T H for the V update (FP64).
//   3. k_als_vg3: every block reduces the Lemma 2 partials and forms the V
//      update itself (CV = g (W^T W * H^T H)^-1 in FP64, normalised through
//      D^T D, rounded, Psi and V^T V from the rounded CV), inverts
//      V^T V * H^T H (FP64), then its share
//      of the W update W_k = G3_k Ginv (FP64), of W^T W and of the
//      convergence value e = sum_k ||Pi_k - H S_k CV^T||^2 (double-float).
// Every block computes the same update from the same partials in the same
// order, so all blocks hold identical H, CV and inverses; block 0 writes them
// for the launches that follow.  The single-block update kernels of the
// five-launch iteration (k_update_h, k_update_v) thereby leave the critical
// path: their reductions and FP64 products now run in every block of the
// grid that needs their result.
#include "common.cuh"
#include "internal.h"
#include "als_phases.cuh"
#include "small_solve.cuh"

namespace dp2 {

// Blocks and warps of the two grids: one block per SM at most, as many warps
// (<= 16) as the per-warp shared memory allows.
static int a3_warps(int R) {
  const int per = (2 * R * R + 3 * R * R + 2 * R) * 4;  // slots (2 RR) + per-warp scratch
  int w = (96 * 1024) / per;
  return w < 1 ? 1 : (w > 16 ? 16 : w);
}

// The Lemma 2 grid launches one extra block (the V update's factor): at most
// num_sms - 1 regular blocks keep both grids within one wave of one block per SM.
int als3_blocks(int K, int R, int num_sms) {
  const int nw = a3_warps(R);
  const int want = (K + nw - 1) / nw;
  return std::max(1, std::min(want, num_sms - 1));
}

// ------------------------------------------------------ H update + Lemma 2 --
// part2[blk] (R x R): g(m, r) = sum over the block's slices of W(k, r)
// sum_i Pi_k(i, m) H(i, r) as double-float sums (hi in [0, RR), lo in
// [RR, 2 RR)): the V update's system has condition numbers up to ~1e8 on
// nearly collinear factors, where FP32 rounding of g that no perturbation of
// the Pi_k explains derails the iteration.  The extra (last) block factors
// InvV = (W^T W * H^T H)^-1 in FP64.
__global__ void k_als_hg2(int K, int R, const float* __restrict__ part1, int nq, int pstride,
                          const double* __restrict__ InvH, const float* __restrict__ Pi, const float* __restrict__ W,
                          const double* __restrict__ WtW, float* __restrict__ Hg, double* __restrict__ HtHg,
                          float* __restrict__ part2, double* __restrict__ InvV, double* __restrict__ Lw,
                          double* __restrict__ Vw, int* __restrict__ status) {
  extern __shared__ __align__(16) double sd[];
  const int RR = R * R, T = blockDim.x;
  const int nw = T >> 5, warp = threadIdx.x >> 5;
  double* red = sd;          // T
  double* G1 = red + T;      // RR
  double* Hn = G1 + RR;      // RR
  double* HtH = Hn + RR;     // RR
  double* Gm = HtH + RR;     // RR
  double* fac = Gm + RR;     // spd_pinv_words(R)
  float* hs = reinterpret_cast<float*>(fac + spd_pinv_words(R));
  float* slots = hs + RR;                       // nw x 2 RR
  float* pks = slots + 2 * nw * RR + warp * RR;  // nw x RR
  block_h_update(part1, nq, pstride, InvH, R, red, G1, Hn, hs, HtH, status);
  if (blockIdx.x == 0)
    for (int e = threadIdx.x; e < RR; e += T) {
      Hg[e] = hs[e];
      HtHg[e] = HtH[e];
    }
  if (blockIdx.x == gridDim.x - 1) {
    // the V update's factor: (W^T W * H^T H)^-1 in FP64
    for (int e = threadIdx.x; e < RR; e += T) Gm[e] = WtW[e] * HtH[e];
    __syncthreads();
    block_spd_pinv<double, double>(Gm, InvV, Lw, Vw, R, fac, status);
    return;
  }
  const int nb = gridDim.x - 1;
  for (int e = threadIdx.x; e < 2 * nw * RR; e += T) slots[e] = 0.f;
  __syncthreads();
  lemma2_warp(K, R, Pi, W, hs, slots + warp * 2 * RR, pks, (int64_t)blockIdx.x * nw + warp, (int64_t)nb * nw, 1);
  __syncthreads();
  block_slots_df(slots, nw, 2 * RR, RR, part2 + (int64_t)blockIdx.x * pstride);
}

// ------------------------------------------------- V update + W update --
// Every block: g from the Lemma 2 partials (double-float halves combined in
// FP64), CV = g InvV (FP64), columns scaled to unit norm through D^T D and
// rounded to FP32, Psi = D^T D CV and V^T V = CV^T D^T D CV from the rounded
// CV, Ginv = (V^T V * H^T H)^-1 in FP64.  Then W_k = G3_k Ginv for
// the block's slices, G3(k, r) = H(:, r)^T Pi_k Psi(:, r) (FP32, insensitive),
// the product in FP64; partials (double-float) of W^T W, from the stored FP32
// W, and of e_k = ||Pi_k - H S_k CV^T||^2 (entries [0, RR) / [RR, 2 RR): W^T W
// hi / lo; 2 RR, 2 RR + 1: e hi / lo).
__global__ void k_als_vg3(int K, int R, const float* __restrict__ part2, int nb2, int pstride,
                          const double* __restrict__ InvV, const double* __restrict__ DtD,
                          const double* __restrict__ HtHg, const float* __restrict__ Hg, const float* __restrict__ Pi,
                          float* __restrict__ CVg, double* __restrict__ Psig, double* __restrict__ VtVg,
                          double* __restrict__ Ginvg, float* __restrict__ W, float* __restrict__ part3,
                          int* __restrict__ status) {
  extern __shared__ __align__(16) double sd[];
  __shared__ float ered[32][2];
  const int RR = R * R, T = blockDim.x;
  const int nw = T >> 5, warp = threadIdx.x >> 5;
  double* red = sd;          // T
  double* Cb = red + T;      // 2 RR: reduced hi / lo halves
  double* C = Cb + 2 * RR;   // RR
  double* DC = C + RR;       // RR
  double* Gm = DC + RR;      // RR
  double* gi = Gm + RR;      // RR: Ginv
  double* fac = gi + RR;     // spd_pinv_words(R)
  double* Lw = fac + spd_pinv_words(R);  // RR: work arrays of the pseudoinverse
  double* Vw = Lw + RR;                       // fallback, private to the block
  float* ps = reinterpret_cast<float*>(Vw + RR);
  float* hs = ps + RR;
  float* cvs = hs + RR;
  float* slots = cvs + RR;                             // nw x 2 RR
  float* pks = slots + 2 * nw * RR + warp * (RR + 2 * R);
  float* g3 = pks + RR;
  float* wn = g3 + R;

  // ---- V update (Lemma 2), the same in every block
  for (int e = threadIdx.x; e < RR; e += T) hs[e] = Hg[e];
  block_v_update(part2, nb2, pstride, InvV, DtD, HtHg, R, red, Cb, C, DC, Gm, cvs, ps,
                 blockIdx.x == 0 ? VtVg : nullptr, CVg, Psig, status);
  block_spd_pinv<double, double>(Gm, gi, Lw, Vw, R, fac, status);
  if (blockIdx.x == 0)
    for (int e = threadIdx.x; e < RR; e += T) Ginvg[e] = gi[e];

  // ---- Lemma 3 and the W update for this block's slices
  for (int e = threadIdx.x; e < nw * 2 * RR; e += T) slots[e] = 0.f;
  __syncthreads();
  DF ek = {0.f, 0.f};
  lemma3_warp(K, R, Pi, ps, hs, cvs, gi, W, slots + warp * 2 * RR, pks, g3, wn, ek, (int64_t)blockIdx.x * nw + warp,
              (int64_t)gridDim.x * nw, 1);
  __syncthreads();
  block_lemma3_out(slots, nw, 2 * RR, R, ek, ered, part3 + (int64_t)blockIdx.x * pstride);
}

// ---------------------------------------------------------------- launchers --
static size_t hg2_smem(int R, int T, int nw) {
  const size_t RR = (size_t)R * R;
  return (T + 4 * RR + spd_pinv_words(R)) * sizeof(double) + (RR + 2 * nw * RR + nw * RR) * sizeof(float);
}
static size_t vg3_smem(int R, int T, int nw) {
  const size_t RR = (size_t)R * R;
  return (T + 8 * RR + spd_pinv_words(R)) * sizeof(double) +
         (3 * RR + 2 * nw * RR + nw * (RR + 2 * R)) * sizeof(float);
}

bool als3_supported(int R) { return R <= 32; }

// One iteration = 3 launches: the Q-step grid (its extra block closes the
// previous iteration and factors the H update's matrix), k_als_hg2 (H update
// in every block, Lemma 2 partials, extra block: the V update's factor),
// k_als_vg3 (V update and W-update inverse in every block, Lemma 3, W, the
// partials of W^T W and e).
void launch_als_iteration3(AlsBufs& b, int it, cudaStream_t s) {
  const int R = b.R, RR = R * R, ps = 2 * RR + 2;
  const int nw = a3_warps(R), T = nw * 32;
  float* p1 = b.part;
  float* p2 = b.part + (size_t)b.pr * ps;
  float* p3 = b.part + (size_t)2 * b.pr * ps;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_als_hg2, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_als_vg3, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr = true;
  }
  PreSolve ph;
  ph.R = R;
  ph.part3 = it > 0 ? p3 : nullptr;
  ph.nparts = b.nblk;
  ph.pstride = ps;
  ph.it = it;
  ph.WtW = b.WtW;
  ph.B = b.VtV;
  ph.loss = b.loss;
  ph.Inv = b.InvH;
  ph.L = b.small;
  ph.V = b.small + RR;
  ph.status = b.status;
  launch_qstep_reg(b, p1, ps, 1, s, &ph);
  DP2_COUNTED(k_als_hg2<<<b.nblk + 1, T, hg2_smem(R, T, nw), s>>>(b.K, R, p1, b.nq, ps, b.InvH, b.Pi, b.W, b.WtW, b.H,
                                                                  b.HtH, p2, b.InvV, b.small, b.small + RR,
                                                                  b.status));
  DP2_COUNTED(k_als_vg3<<<b.nblk, T, vg3_smem(R, T, nw), s>>>(b.K, R, p2, b.nblk, ps, b.InvV, b.DtD, b.HtH, b.H,
                                                              b.Pi, b.CV, b.Psi, b.VtV, b.Ginv, b.W, p3,
                                                              b.status));
}

}  // namespace dp2
