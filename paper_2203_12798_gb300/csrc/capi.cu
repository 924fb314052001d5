// C ABI of libdpar2: argument checks, scratch management and the launch
// sequence of the two-stage compression (Sec. III-B) and of the ALS
// iterations (Alg. 3).  Every numerical step runs in the kernels of this
// library; the host only validates, allocates, launches and reads back the
// status word and the requested scalars.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"
#include "internal.h"

using namespace dp2;

namespace dp2 {
// Kernels enqueued by this library since it was loaded (all contexts and
// threads).  Launches recorded into a CUDA graph are taken back out when the
// capture ends and counted again each time the graph is launched.
std::atomic<long long> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
}  // namespace dp2

namespace {

struct Fail {
  dpar2_status st;
  std::string msg;
};

inline void ck(cudaError_t e, const char* what) {
  if (e != cudaSuccess) {
    cudaGetLastError();
    throw Fail{e == cudaErrorMemoryAllocation ? DPAR2_ERR_OOM : DPAR2_ERR_CUDA,
               std::string(what) + ": " + cudaGetErrorString(e)};
  }
}
#define CK(x) ck((x), #x)

inline void require(bool c, dpar2_status st, const std::string& msg) {
  if (!c) throw Fail{st, msg};
}

template <typename T>
T* wsget(dpar2_ctx* ctx, const char* name, size_t count) {
  void* p = ctx->get(name, count * sizeof(T));
  if (!p) throw Fail{DPAR2_ERR_OOM, std::string("cannot allocate scratch '") + name + "'"};
  return static_cast<T*>(p);
}

inline cudaStream_t work_stream(dpar2_ctx* ctx) {
  return reinterpret_cast<cudaStream_t>(ctx->ws["__work_stream"].p);
}

// Buffer of a compression object: from the owner's stream-ordered pool on its
// work stream (no device-wide synchronisation, memory reused across objects),
// else plain cudaMalloc.
void release(dpar2_comp* c, dp2::DevBuf& b) {
  if (!b.p) return;
  if (c->owner && c->owner->pool) cudaFreeAsync(b.p, work_stream(c->owner));
  else cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
}

void alloc(dpar2_comp* c, dp2::DevBuf& b, size_t bytes) {
  release(c, b);
  if (bytes == 0) return;
  cudaError_t e = (c->owner && c->owner->pool)
                      ? cudaMallocFromPoolAsync(&b.p, bytes, c->owner->pool, work_stream(c->owner))
                      : cudaMalloc(&b.p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    b.p = nullptr;
    throw Fail{DPAR2_ERR_OOM, "device allocation of " + std::to_string(bytes) + " bytes failed"};
  }
  b.bytes = bytes;
}

// Frees what the context holds; the work stream and the pool stay while
// compression objects made by it are alive (the last one's free finishes).
void ctx_release(dpar2_ctx* ctx) {
  cudaDeviceSynchronize();
  for (auto& kv : ctx->ws) {
    if (!kv.second.p || kv.first == "__work_stream") continue;
    if (kv.first == "__event" || kv.first.rfind("__copy_ev", 0) == 0)
      cudaEventDestroy(reinterpret_cast<cudaEvent_t>(kv.second.p));
    else if (kv.first.rfind("__copy_stream", 0) == 0) cudaStreamDestroy(reinterpret_cast<cudaStream_t>(kv.second.p));
    else cudaFree(kv.second.p);
    kv.second.p = nullptr;
  }
  for (int i = 0; i < 2 * DPAR2_NUM_PHASES; ++i)
    if (ctx->tev[i]) cudaEventDestroy(ctx->tev[i]), ctx->tev[i] = nullptr;
  if (ctx->d_status) cudaFree(ctx->d_status), ctx->d_status = nullptr;
  if (ctx->h_status) cudaFreeHost(ctx->h_status), ctx->h_status = nullptr;
  if (ctx->hstage) cudaFreeHost(ctx->hstage), ctx->hstage = nullptr;
  if (ctx->live_comps > 0) {
    ctx->closing = true;
    return;
  }
  if (ctx->ws["__work_stream"].p) cudaStreamDestroy(work_stream(ctx));
  if (ctx->pool) cudaMemPoolDestroy(ctx->pool);
  delete ctx;
}

size_t dtype_size(dpar2_dtype dt) { return dt == DPAR2_F32 ? 4 : 2; }

// n int64 values host -> device through the context's pinned staging area, so
// that the copy is asynchronous (a copy from pageable memory waits for the
// stream first).  The area grows (after draining the stream) when a call needs more.
void h2d_bytes(dpar2_ctx* ctx, void* dst, const void* src, size_t bytes, cudaStream_t s) {
  const size_t n = (bytes + 7) / 8;  // staging words
  if (ctx->hstage_used + n > ctx->hstage_cap) {
    CK(cudaStreamSynchronize(s));
    if (ctx->hstage) cudaFreeHost(ctx->hstage);
    ctx->hstage = nullptr;
    ctx->hstage_cap = std::max<size_t>(2 * (ctx->hstage_used + n), 1 << 16);
    ctx->hstage_used = 0;
    if (cudaMallocHost(&ctx->hstage, ctx->hstage_cap * sizeof(int64_t)) != cudaSuccess) {
      cudaGetLastError();
      ctx->hstage = nullptr;
      ctx->hstage_cap = 0;
      throw Fail{DPAR2_ERR_OOM, "pinned host allocation failed"};
    }
  }
  int64_t* h = ctx->hstage + ctx->hstage_used;
  ctx->hstage_used += n;
  std::memcpy(h, src, bytes);
  CK(cudaMemcpyAsync(dst, h, bytes, cudaMemcpyHostToDevice, s));
}

void h2d_i64(dpar2_ctx* ctx, int64_t* dst, const int64_t* src, size_t n, cudaStream_t s) {
  h2d_bytes(ctx, dst, src, n * sizeof(int64_t), s);
}

// The projection's slice-to-CTA schedule for this call: 0 round-robin, 1
// longest-slices-first work lists (copied to the device here).  opt_schedule
// -1 takes the choice stored for this problem shape, if any (-1 = not tuned).
struct ProjSched {
  int choice = 0;
  const int* lptr = nullptr;
  const int* items = nullptr;
  int nlists = 0;
};

std::string tune_key(int K, int J, int ell, dpar2_dtype dt, int64_t N, int64_t maxI) {
  return "pj:" + std::to_string(K) + ":" + std::to_string(J) + ":" + std::to_string(ell) + ":" +
         std::to_string((int)dt) + ":" + std::to_string(N) + ":" + std::to_string(maxI);
}

ProjSched proj_sched(dpar2_ctx* ctx, int choice, const int64_t* row_offsets, int K, int nJb, const std::string& key,
                     cudaStream_t s) {
  ProjSched ps;
  ps.choice = choice;
  if (choice != 1) return ps;
  ps.nlists = ctx->num_sms;
  const size_t nl = (size_t)ps.nlists + 1, ni = (size_t)K * nJb;
  int* d_lptr = wsget<int>(ctx, "pj_lptr", nl);
  int* d_items = wsget<int>(ctx, "pj_items", ni);
  // the lists on the device are those of the last problem shape that used them
  const std::string lkey = key + ":" + std::to_string(nJb) + ":" + std::to_string(ps.nlists);
  if (ctx->pj_lists_key != lkey) {
    std::vector<int> lptr, items;
    project_lpt_lists(row_offsets, K, nJb, ps.nlists, lptr, items);
    h2d_bytes(ctx, d_lptr, lptr.data(), lptr.size() * sizeof(int), s);
    h2d_bytes(ctx, d_items, items.data(), items.size() * sizeof(int), s);
    ctx->pj_lists_key = lkey;
  }
  ps.lptr = d_lptr;
  ps.items = d_items;
  return ps;
}

// Runs `body` with the context's device current and a private work stream
// ordered after `user` work; converts failures into status codes.
template <typename F>
dpar2_status guarded(dpar2_ctx* ctx, void* user_stream, F&& body) {
  if (!ctx || ctx->closing) return DPAR2_ERR_INVALID_ARG;
  ctx->err.clear();
  int prev = -1;
  cudaGetDevice(&prev);
  try {
    CK(cudaSetDevice(ctx->device));
    cudaStream_t us = static_cast<cudaStream_t>(user_stream);
    cudaStream_t work = reinterpret_cast<cudaStream_t>(ctx->ws["__work_stream"].p);
    cudaEvent_t ev = reinterpret_cast<cudaEvent_t>(ctx->ws["__event"].p);
    CK(cudaEventRecord(ev, us));
    CK(cudaStreamWaitEvent(work, ev, 0));
    CK(cudaMemsetAsync(ctx->d_status, 0, sizeof(int), work));
    ctx->hstage_used = 0;
    body(work);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(ctx->h_status, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, work));
    CK(cudaStreamSynchronize(work));
    for (int ph = 0; ph < DPAR2_NUM_PHASES; ++ph) {
      if (!ctx->tpending[ph]) continue;
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, ctx->tev[2 * ph], ctx->tev[2 * ph + 1]) == cudaSuccess) ctx->tms[ph] = ms;
      cudaGetLastError();
      ctx->tpending[ph] = false;
    }
    const int st = *ctx->h_status;
    if (st & ST_TIMEOUT) throw Fail{DPAR2_ERR_TIMEOUT, "a bounded device-side wait gave up"};
    if (st & ST_NONFINITE) throw Fail{DPAR2_ERR_NUMERICAL, "non-finite values met on the device"};
  } catch (const Fail& f) {
    ctx->err = f.msg;
    if (prev >= 0) cudaSetDevice(prev);
    return f.st;
  }
  if (prev >= 0) cudaSetDevice(prev);
  return DPAR2_OK;
}

inline void tbegin(dpar2_ctx* c, cudaStream_t s, int ph) {
  if (c->timing) cudaEventRecord(c->tev[2 * ph], s);
}
inline void tend(dpar2_ctx* c, cudaStream_t s, int ph) {
  if (c->timing) {
    cudaEventRecord(c->tev[2 * ph + 1], s);
    c->tpending[ph] = true;
  }
}

// Row splits of a Gram so that at least ~2 blocks per SM work on it.
int gram_splits(int K, int64_t maxI) {
  if (K >= 256) return 1;
  const int64_t want = (300 + K - 1) / K;
  return (int)std::max<int64_t>(1, std::min<int64_t>(want, (maxI + 255) / 256));
}

// CholeskyQR2 of the per-slice sketches Y (rows x LP, in place): after the
// call Y holds Q1 = Y R1^+ and M2 = R2^+ with Q = Q1 M2 column-orthonormal on
// its numerical rank.  Both Grams are double-float sums of exact products
// (about 48 significant bits) stored in FP64: an FP32 sum of the second Gram
// over I_k rows is off by ~sqrt(I_k) eps32 (4e-6 at 4000 rows), more than the
// departure of Q1 from orthonormality it is there to measure.  First step:
// FP64 Cholesky; second step, whose matrix is within ~1e-6 of the identity:
// FP32 Cholesky (relative accuracy eps32 for a matrix of condition ~1);
// dependent columns dropped.
void cholqr2(dpar2_ctx* ctx, float* Y, const int64_t* d_off, int K, int64_t maxI, int ell, int LP, float* M2,
             int* rank, cudaStream_t s, const char* tag) {
  std::string t(tag);
  double* G = wsget<double>(ctx, (t + "_G").c_str(), (size_t)K * LP * LP);
  float* M1 = wsget<float>(ctx, (t + "_M1").c_str(), (size_t)K * LP * LP);
  const int nsplit = gram_splits(K, maxI);
  double* Gp = nsplit > 1 ? wsget<double>(ctx, (t + "_Gp").c_str(), (size_t)K * nsplit * LP * LP) : nullptr;
  launch_gram_dd(Y, LP, d_off, K, ell, G, Gp, nsplit, s);
  launch_chol_drop(G, K, ell, LP, 1e-11, M1, nullptr, ctx->d_status, true, s);
  launch_formq_gram(Y, LP, d_off, K, ell, M1, G, Gp, nsplit, s);
  launch_chol_drop(G, K, ell, LP, 1e-6, M2, rank, ctx->d_status, false, s);
}

__global__ void k_b1_to_omk(const float* __restrict__ B1, int K, int ell, int LP, int J, int Jp, int Jpad,
                            float* __restrict__ omk) {
  const int64_t n = (int64_t)K * Jpad * LP;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = i / ((int64_t)Jpad * LP);
    const int rem = (int)(i % ((int64_t)Jpad * LP));
    const int j = rem / LP, c = rem % LP;
    omk[i] = (j < J && c < ell) ? B1[(k * LP + c) * Jp + j] : 0.f;
  }
}

__global__ void k_apply_m2(float* __restrict__ Y, const int64_t* __restrict__ off, int LP,
                           const float* __restrict__ M2) {
  // Y_k <- Y_k M2_k row by row (generic LP, used once per power iteration)
  const int k = blockIdx.y;
  const int64_t row = off[k] + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= off[k + 1]) return;
  float y[kMaxEll];
  for (int c = 0; c < LP; ++c) y[c] = Y[row * LP + c];
  const float* m = M2 + (int64_t)k * LP * LP;
  for (int c = 0; c < LP; ++c) {
    float s = 0.f;
    for (int i = 0; i < LP; ++i) s = fmaf(y[i], m[i * LP + c], s);
    Y[row * LP + c] = s;
  }
}

__global__ void k_sum_f64(const double* __restrict__ v, int n, double* __restrict__ out) {
  __shared__ double red[256];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += 256) s += v[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = red[0];
}

// Stage 1 of the compression (Alg. 1 for every slice; the first loop of
// Alg. 3) on the slices k0 .. k0 + Kc - 1, whose rows start at X (row 0 is
// the first row of slice k0, row pitch ldx): the sketch, CholeskyQR2 (and the
// power iterations), the projection with ||X_k||^2, the small SVDs, the
// blocks C_k B_k of M and A_k.  off: host offsets of those slices relative to
// their first row (Kc + 1), d_off the same on the device.  Writes the
// compression's A rows, B_k, M blocks, ||X_k||^2 and ranks of these slices;
// scratch is the context's (sized for this range).  Every slice is computed
// the same way whatever range it is part of, except for the Gram row splits
// of ranges shorter than 256 slices (a different summation order).
void stage1_range(dpar2_ctx* ctx, dpar2_comp* comp, const void* X, int64_t ldx, dpar2_dtype dtype,
                  const dpar2_options* opt, int k0, int Kc, const int64_t* off, const int64_t* d_off,
                  const float* om_pad, bool timed, cudaStream_t s) {
  const int J = comp->J, R = comp->R, ell = comp->ell, LP = comp->LP;
  const int Jp = round_up(J, 4), Jpad = round_up(J, 32);
  const int64_t N = off[Kc];
  int64_t maxI = 0;
  for (int k = 0; k < Kc; ++k) maxI = std::max<int64_t>(maxI, off[k + 1] - off[k]);
  const size_t es = dtype_size(dtype);
  int* rank1 = static_cast<int*>(comp->rank1.p) + k0;
  double* xn2 = static_cast<double*>(comp->xnorm2.p) + k0;
  float* Bk = static_cast<float*>(comp->Bk.p) + (size_t)k0 * R;
  void* Mb = static_cast<__nv_bfloat16*>(comp->M.p) + (size_t)k0 * R * comp->Jq;
  const int64_t mpart = (int64_t)comp->K * R * comp->Jq;
  float* Aout = static_cast<float*>(comp->A.p) + (size_t)comp->h_offsets[k0] * R;
  auto tb = [&](int ph) { if (timed) tbegin(ctx, s, ph); };
  auto te = [&](int ph) { if (timed) tend(ctx, s, ph); };
  // ---- sketch Y = X Omega (pass 1 over X) ----
  float* Y = wsget<float>(ctx, "Y", (size_t)N * LP);
  float* M2 = wsget<float>(ctx, "M2", (size_t)Kc * LP * LP);
  float* B1 = wsget<float>(ctx, "B1", (size_t)Kc * LP * Jp);
  const int nJb = project_blocks(Jp, LP);
  double* xpart = wsget<double>(ctx, "xpart", (size_t)Kc * nJb);
  // tensor-core path: 16-bit X, all slices in one persistent launch
  const bool use_tc = dtype != DPAR2_F32 && !(opt->flags & (DPAR2_FLAG_GENERIC | DPAR2_FLAG_PER_SLICE)) &&
                      tc_available();
  const int LPN = tc_lpn(ell);
  void* omT16 = nullptr;
  if (use_tc) {
    omT16 = wsget<uint16_t>(ctx, "omT16", (size_t)LPN * Jpad);
    launch_omega_t16(om_pad, Jpad, LP, LPN, dtype, omT16, s);
  }
  tb(DPAR2_PH_SKETCH);
  bool sketched = false;
  if (use_tc)
    sketched = launch_sketch_tc(X, dtype, ldx, N, J, omT16, Jpad, LPN, LP, Y, ctx->num_sms, ctx->d_status, s);
  if (sketched) {
  } else if (opt->flags & DPAR2_FLAG_PER_SLICE) {
    for (int k = 0; k < Kc; ++k) {
      const int64_t r0 = off[k], nk = off[k + 1] - r0;
      launch_sketch_generic(static_cast<const char*>(X) + r0 * ldx * es, dtype, ldx, nk, J, om_pad, LP,
                            Y + r0 * LP, s);
    }
  } else {
    launch_sketch_generic(X, dtype, ldx, N, J, om_pad, LP, Y, s);
  }
  te(DPAR2_PH_SKETCH);
  tb(DPAR2_PH_QR);
  cholqr2(ctx, Y, d_off, Kc, maxI, ell, LP, M2, rank1, s, "s1");
  // tensor-core projection operands: Q1 split into three exact-sum 16-bit
  // parts, slices padded to 64 rows; one partial ||X_k||^2 per (slice,
  // column block, norm warp)
  std::vector<int64_t> hp, htoff;
  int64_t maxPad = 0;
  ProjSched pj;  // the projection's slice-to-CTA schedule for its first candidate
  const std::string tkey = tune_key(Kc, J, ell, dtype, N, maxI);
  int64_t* d_poff = nullptr;
  void* Qs = nullptr;
  double* xp = nullptr;
  int PNS = 0, POFF = 0;  // layout of the projection's Q operand
  proj_layout(ell, &PNS, &POFF);
  // (schedule, work-item width) pairs of the projection: the options' fixed
  // pair, the pair tuned before for this problem shape, or every candidate
  // (both schedules, both widths unless one is given) timed on this call
  auto njb_of = [&](int hv) { return (Jp + project_tc_cols(PNS, hv) - 1) / project_tc_cols(PNS, hv); };
  const int hv_fixed = opt->proj_cols / 128;
  const std::string tkey_w = tkey + ":w" + std::to_string(hv_fixed);
  std::vector<std::pair<int, int>> pj_cand;
  if (opt->schedule >= 0) {
    pj_cand.push_back({opt->schedule > 1 ? 0 : opt->schedule, hv_fixed ? hv_fixed : project_hv_default(PNS)});
  } else {
    auto it = ctx->tuned.find(tkey_w);
    if (it != ctx->tuned.end()) {
      pj_cand.push_back({it->second & 1, it->second >> 1});
    } else {
      for (int sch = 0; sch < 2; ++sch) {
        if (hv_fixed) {
          pj_cand.push_back({sch, hv_fixed});
        } else {
          pj_cand.push_back({sch, project_hv_default(PNS)});
          if (project_hv_alt(PNS)) pj_cand.push_back({sch, project_hv_alt(PNS)});
        }
      }
    }
  }
  int nJb_max = 0;
  for (auto& c : pj_cand) nJb_max = std::max(nJb_max, njb_of(c.second));
  const int pj_hv0 = pj_cand[0].second, nJb_tc = njb_of(pj_hv0);
  if (use_tc) {
    hp.assign(Kc + 1, 0);
    for (int k = 0; k < Kc; ++k) {
      const int64_t pk = round_up64(off[k + 1] - off[k], 64);
      hp[k + 1] = hp[k] + pk;
      maxPad = std::max(maxPad, pk);
    }
    d_poff = wsget<int64_t>(ctx, "poff", (size_t)Kc + 1);
    h2d_i64(ctx, d_poff, hp.data(), (Kc + 1), s);
    Qs = wsget<uint16_t>(ctx, "Qs", (size_t)PNS * hp[Kc]);
    xp = wsget<double>(ctx, "xpart_tc", (size_t)Kc * nJb_max * kProjNormWarps);
    pj = proj_sched(ctx, pj_cand[0].first, off, Kc, nJb_tc, tkey, s);
  }
  // ---- power iterations Y <- X (X^T Q), re-orthonormalised ----
  int64_t* d_toff = nullptr;
  if (use_tc && opt->q > 0) {
    htoff.assign(Kc + 1, 0);
    for (int k = 0; k < Kc; ++k) htoff[k + 1] = htoff[k] + (off[k + 1] - off[k] + 127) / 128;
    d_toff = wsget<int64_t>(ctx, "toff", (size_t)Kc + 1);
    h2d_i64(ctx, d_toff, htoff.data(), (Kc + 1), s);
  }
  for (int it = 0; it < opt->q; ++it) {
    if (use_tc) {
      // B1 = Q1^T X, then Y_k = X_k B1_k^T on the tensor cores: X_k X_k^T Q_k =
      // X_k B1_k^T M2_k up to the upper-triangular M2_k (and the power-of-two
      // row scales of the operand), which leave the next CholeskyQR2's Q unchanged
      launch_qsplit(Y, LP, PNS, POFF, d_off, d_poff, Kc, hp[Kc], maxPad, dtype, Qs, s);
      bool ok = launch_project_tc(X, dtype, ldx, N, d_off, d_poff, Kc, J, Jp, Qs, hp[Kc], PNS, POFF, LP, B1, xp, nJb_tc, true,
                                  ctx->num_sms, ctx->d_status, s, pj.lptr, pj.items, pj.nlists, pj_hv0);
      require(ok, DPAR2_ERR_CUDA, "tensor map encoding failed");
      void* Ms = wsget<uint16_t>(ctx, "Ms", (size_t)Kc * 3 * LPN * Jpad);
      launch_sl_rowsplit(B1, Kc, Jp, J, Jpad, ell, LP, LPN, dtype, Ms, nullptr,
                         wsget<float>(ctx, "Ms_scale", (size_t)Kc * LP), s);
      ok = launch_sketch_seg_tc(X, dtype, ldx, N, J, d_off, d_toff, htoff[Kc], Kc, Ms, Jpad, LPN, LP, Y,
                                ctx->num_sms, ctx->d_status, s);
      require(ok, DPAR2_ERR_CUDA, "tensor map encoding failed");
    } else {
      DP2_COUNTED(k_apply_m2<<<dim3((unsigned)((maxI + 127) / 128), Kc), 128, 0, s>>>(Y, d_off, LP, M2));
      launch_project_generic(X, dtype, ldx, d_off, Kc, J, Jp, Y, LP, B1, nullptr, nullptr, s);
      float* omk = wsget<float>(ctx, "omk", (size_t)Kc * Jpad * LP);
      DP2_COUNTED(k_b1_to_omk<<<4096, 256, 0, s>>>(B1, Kc, ell, LP, J, Jp, Jpad, omk));
      launch_sketch_generic_per_slice(X, dtype, ldx, d_off, Kc, (int)maxI, J, omk, Jpad, LP, Y, s);
    }
    cholqr2(ctx, Y, d_off, Kc, maxI, ell, LP, M2, rank1, s, "s1");
  }

  te(DPAR2_PH_QR);
  // ---- projection B1 = Q1^T X (pass 2 over X) and ||X_k||^2 ----
  int nJb_used = nJb;
  bool projected = false;
  if (use_tc) {
    const int64_t Npad = hp[Kc];
    launch_qsplit(Y, LP, PNS, POFF, d_off, d_poff, Kc, Npad, maxPad, dtype, Qs, s);
    tb(DPAR2_PH_PROJECT);
    int nJb_last = nJb_tc;
    if (pj_cand.size() > 1) {
      // autotune: time every candidate on this call's projection (the same B1;
      // ||X_k||^2 partials laid out per width) and keep the fastest pair for
      // this problem shape
      const int nc = (int)pj_cand.size();
      std::vector<cudaEvent_t> ev(nc + 1);
      for (auto& e : ev) CK(cudaEventCreate(&e));
      CK(cudaEventRecord(ev[0], s));
      for (int c = 0; c < nc; ++c) {
        const ProjSched cs = proj_sched(ctx, pj_cand[c].first, off, Kc, njb_of(pj_cand[c].second), tkey, s);
        projected = launch_project_tc(X, dtype, ldx, N, d_off, d_poff, Kc, J, Jp, Qs, Npad, PNS, POFF, LP, B1, xp,
                                      njb_of(pj_cand[c].second), true, ctx->num_sms, ctx->d_status, s, cs.lptr,
                                      cs.items, cs.nlists, pj_cand[c].second);
        CK(cudaEventRecord(ev[c + 1], s));
      }
      CK(cudaEventSynchronize(ev[nc]));
      int best = 0;
      float tbest = 0.f;
      for (int c = 0; c < nc; ++c) {
        float t = 0.f;
        CK(cudaEventElapsedTime(&t, ev[c], ev[c + 1]));
        if (c == 0 || t < tbest) {
          tbest = t;
          best = c;
        }
      }
      for (auto& e : ev) cudaEventDestroy(e);
      ctx->tuned[tkey_w] = pj_cand[best].first + 2 * pj_cand[best].second;
      ctx->pj_last_schedule = pj_cand[best].first;
      ctx->pj_last_cols = project_tc_cols(PNS, pj_cand[best].second);
      nJb_last = njb_of(pj_cand[nc - 1].second);
      if (pj_cand[best].second != pj_cand[nc - 1].second) {
        // the ||X_k||^2 partials are laid out per work item (their FP64 total
        // follows the width at the FP64 rounding level): leave those of the
        // chosen width, as later calls of this shape will
        const ProjSched cs = proj_sched(ctx, pj_cand[best].first, off, Kc, njb_of(pj_cand[best].second), tkey, s);
        projected = launch_project_tc(X, dtype, ldx, N, d_off, d_poff, Kc, J, Jp, Qs, Npad, PNS, POFF, LP, B1, xp,
                                      njb_of(pj_cand[best].second), true, ctx->num_sms, ctx->d_status, s, cs.lptr,
                                      cs.items, cs.nlists, pj_cand[best].second);
        nJb_last = njb_of(pj_cand[best].second);
      }
    } else {
      projected = launch_project_tc(X, dtype, ldx, N, d_off, d_poff, Kc, J, Jp, Qs, Npad, PNS, POFF, LP, B1, xp, nJb_tc,
                                    true, ctx->num_sms, ctx->d_status, s, pj.lptr, pj.items, pj.nlists, pj_hv0);
      ctx->pj_last_schedule = pj_cand[0].first;
      ctx->pj_last_cols = project_tc_cols(PNS, pj_hv0);
    }
    if (projected) {
      xpart = xp;
      nJb_used = nJb_last * kProjNormWarps;
    }
  } else {
    tb(DPAR2_PH_PROJECT);
    ctx->pj_last_schedule = -1;
    ctx->pj_last_cols = 0;
  }
  if (projected) {
  } else if (opt->flags & DPAR2_FLAG_PER_SLICE) {
    for (int k = 0; k < Kc; ++k)
      launch_project_generic(X, dtype, ldx, d_off + k, 1, J, Jp, Y, LP, B1 + (size_t)k * LP * Jp,
                             xpart + (size_t)k * nJb, nullptr, s);
  } else {
    launch_project_generic(X, dtype, ldx, d_off, Kc, J, Jp, Y, LP, B1, xpart, nullptr, s);
  }
  te(DPAR2_PH_PROJECT);
  tb(DPAR2_PH_SMALL);
  launch_reduce_rows_f64(xpart, Kc, nJb_used, xn2, s);

  // ---- small SVD of B = M2^T B1 -> C_k B_k blocks of M, T_k, A_k ----
  double* GB = wsget<double>(ctx, "GB", (size_t)Kc * LP * LP);
  float* T = wsget<float>(ctx, "T", (size_t)Kc * LP * R);
  launch_gram_b1(B1, Jp, J, Kc, ell, LP, GB, s);
  launch_eig_top(GB, M2, Kc, ell, LP, R, T, nullptr, ctx->d_status, s);
  launch_mblock(B1, Jp, J, Kc, ell, LP, R, T, Bk, Mb, mpart, comp->Jq, rank1, 1e-5f, s);
  launch_seg_product(Y, LP, LP, T, (int64_t)LP * R, R, Aout, R, d_off, Kc, maxI, s);

  te(DPAR2_PH_SMALL);
}

// Stage 2 of the compression (Sec. III-B, the randomized SVD of
// M = [C_1 B_1 ... C_K B_K], J x KR): D, E, F~_k = F^(k) E and D^T D of the
// compression from its M blocks.
void stage2_all(dpar2_ctx* ctx, dpar2_comp* comp, const dpar2_options* opt, const float* omega2, cudaStream_t s) {
  const int K = comp->K, J = comp->J, R = comp->R, ell = comp->ell, LP = comp->LP;
  // ---- stage 2: randomized SVD of M (J x KR) ----
  tbegin(ctx, s, DPAR2_PH_STAGE2);
  const int64_t KR = (int64_t)K * R;
  const float* om2 = omega2;
  if (!om2) {
    float* g = wsget<float>(ctx, "omega2", (size_t)KR * ell);
    launch_gaussian(opt->seed, 1, KR * ell, g, 1, s);
    om2 = g;
  }
  float* om2p = wsget<float>(ctx, "om2_pad", (size_t)KR * LP);
  launch_pad_omega(om2, (int)KR, ell, (int)KR, LP, DPAR2_F32, om2p, s);
  // tensor-core passes over the BF16 parts of M^T; right operands split the same way
  const void* Ms = comp->M.p;
  const int Jq = comp->Jq;
  const int64_t KRq = round_up64(KR, 64);
  const int NB = s2_nb(LP);
  void* bsk = wsget<uint16_t>(ctx, "s2_bsk", (size_t)NB * KRq);
  void* bpj = wsget<uint16_t>(ctx, "s2_bpj", (size_t)NB * Jq);
  const int nchS = s2_tc_chunks(true, KR, J, Jq, ctx->num_sms);
  const int nchP = s2_tc_chunks(false, KR, J, Jq, ctx->num_sms);
  float* Y2p = wsget<float>(ctx, "Y2p", (size_t)nchS * J * LP);
  float* Y2 = wsget<float>(ctx, "Y2", (size_t)J * LP);
  float* B2pp = wsget<float>(ctx, "B2pp", (size_t)nchP * KR * LP);
  float* B2p = wsget<float>(ctx, "B2p", (size_t)KR * LP);
  // Y2 = M F (F: KR x LP)
  auto sketch = [&](const float* F) {
    launch_s2_split_rhs(F, KR, LP, KRq, bsk, s);
    require(launch_s2_tc(true, Ms, KR, J, Jq, bsk, KRq, LP, Y2p, nchS, ctx->num_sms, ctx->d_status, s),
            DPAR2_ERR_CUDA, "tensor map encoding failed");
    launch_sum_parts(Y2p, nchS, (int64_t)J * LP, Y2, s);
  };
  // B2p = M^T G (G: J x LP)
  auto project = [&](const float* G) {
    launch_s2_split_rhs(G, J, LP, Jq, bpj, s);
    require(launch_s2_tc(false, Ms, KR, J, Jq, bpj, Jq, LP, B2pp, nchP, ctx->num_sms, ctx->d_status, s),
            DPAR2_ERR_CUDA, "tensor map encoding failed");
    launch_sum_parts(B2pp, nchP, KR * LP, B2p, s);
  };
  sketch(om2p);
  int64_t* off2 = wsget<int64_t>(ctx, "off2", 4);
  const int64_t h_off2[4] = {0, (int64_t)J, 0, KR};
  h2d_i64(ctx, off2, h_off2, sizeof(h_off2) / sizeof(int64_t), s);
  float* M2s = wsget<float>(ctx, "M2s", (size_t)LP * LP);
  cholqr2(ctx, Y2, off2, 1, J, ell, LP, M2s, nullptr, s, "s2");
  for (int it = 0; it < opt->q; ++it) {
    // Y2 <- M (M^T Q2)
    DP2_COUNTED(k_apply_m2<<<dim3((unsigned)((J + 127) / 128), 1), 128, 0, s>>>(Y2, off2, LP, M2s));
    project(Y2);
    sketch(B2p);
    cholqr2(ctx, Y2, off2, 1, J, ell, LP, M2s, nullptr, s, "s2");
  }
  project(Y2);
  double* G2 = wsget<double>(ctx, "G2", (size_t)LP * LP);
  {
    const int ns = gram_splits(1, KR);
    double* Gp = wsget<double>(ctx, "G2p", (size_t)ns * LP * LP);
    launch_gram_dd(B2p, LP, off2 + 2, 1, ell, G2, Gp, ns, s);
  }
  float* T2 = wsget<float>(ctx, "T2", (size_t)LP * R);
  launch_eig_top(G2, M2s, 1, ell, LP, R, T2, nullptr, ctx->d_status, s);
  launch_seg_product(Y2, LP, LP, T2, 0, R, static_cast<float*>(comp->D.p), R, off2, 1, J, s);
  launch_seg_product(B2p, LP, LP, T2, 0, R, static_cast<float*>(comp->Ft.p), R, off2 + 2, 1, KR, s);
  {
    double* epart = wsget<double>(ctx, "en_part", (size_t)kEnormBlocks * R);
    float* ekeep = wsget<float>(ctx, "en_keep", (size_t)R);
    int* endrop = wsget<int>(ctx, "en_ndrop", 1);
    launch_s2_enorm(static_cast<float*>(comp->Ft.p), KR, R, static_cast<float*>(comp->D.p), J,
                    static_cast<float*>(comp->E.p), 1e-6f, epart, ekeep, endrop, s);
  }
  launch_atb(J, R, static_cast<const float*>(comp->D.p), static_cast<const float*>(comp->D.p),
             static_cast<double*>(comp->DtD.p), wsget<float>(ctx, "atb_part", (size_t)kAtbBlocks * R * R), s);
  tend(ctx, s, DPAR2_PH_STAGE2);
}

// Argument checks of dpar2_compress / dpar2_compress_host (host only, before
// any launch).  device_x: X is device memory that must be 16-byte aligned.
dpar2_status check_compress(dpar2_ctx* ctx, int K, int J, const int64_t* row_offsets, const void* X, int64_t ldx,
                            dpar2_dtype dtype, const dpar2_options* opt, dpar2_comp** out, bool device_x) {
  try {
    require(out != nullptr, DPAR2_ERR_INVALID_ARG, "out is null");
    *out = nullptr;
    require(opt && X && row_offsets, DPAR2_ERR_INVALID_ARG, "opt, X and row_offsets must be non-null");
    require(dtype == DPAR2_F32 || dtype == DPAR2_BF16 || dtype == DPAR2_F16, DPAR2_ERR_INVALID_ARG, "bad dtype");
    require(K >= 1 && J >= 1, DPAR2_ERR_SHAPE, "K and J must be >= 1");
    require(opt->R >= 1 && opt->R <= kMaxR && opt->R <= J, DPAR2_ERR_SHAPE, "need 1 <= R <= min(J, 64)");
    require(opt->p >= 0 && opt->R + opt->p <= std::min(J, kMaxEll), DPAR2_ERR_SHAPE, "need R + p <= min(J, 64)");
    require(opt->q >= 0 && opt->q <= 8, DPAR2_ERR_INVALID_ARG, "need 0 <= q <= 8");
    {
      int ns = 0, offp = 0;
      proj_layout(opt->R + opt->p, &ns, &offp);
      const int hv = opt->proj_cols / 128;
      require(opt->proj_cols == 0 || (opt->proj_cols % 128 == 0 &&
                                      (hv == project_hv_default(ns) || hv == project_hv_alt(ns))),
              DPAR2_ERR_INVALID_ARG, "proj_cols must be 0 or a work-item width of the projection for this l");
    }
    require(ldx >= J, DPAR2_ERR_SHAPE, "ldx < J");
    require((ldx * (int64_t)dtype_size(dtype)) % 16 == 0, DPAR2_ERR_INVALID_ARG,
            "ldx * sizeof(dtype) must be a multiple of 16 bytes");
    if (device_x)
      require((reinterpret_cast<uintptr_t>(X) & 15) == 0, DPAR2_ERR_INVALID_ARG, "X must be 16-byte aligned");
    require(row_offsets[0] == 0, DPAR2_ERR_SHAPE, "row_offsets[0] must be 0");
    for (int k = 0; k < K; ++k)
      require(row_offsets[k + 1] > row_offsets[k], DPAR2_ERR_SHAPE, "every slice needs I_k >= 1 rows");
    return DPAR2_OK;
  } catch (const Fail& f) {
    ctx->err = f.msg;
    return f.st;
  }
}

// A new compression object for K slices (buffers from the context's pool),
// its device offsets copied.
dpar2_comp* new_comp(dpar2_ctx* ctx, int K, int J, const int64_t* row_offsets, const dpar2_options* opt,
                     cudaStream_t s) {
  const int R = opt->R, ell = opt->R + opt->p, LP = round_up(ell, 8);
  const int64_t N = row_offsets[K];
  int64_t maxI = 0;
  for (int k = 0; k < K; ++k) maxI = std::max<int64_t>(maxI, row_offsets[k + 1] - row_offsets[k]);
  dpar2_comp* comp = new dpar2_comp();
  comp->owner = ctx;
  ++ctx->live_comps;
  comp->K = K;
  comp->J = J;
  comp->R = R;
  comp->ell = ell;
  comp->LP = LP;
  comp->N = N;
  comp->maxI = maxI;
  comp->h_offsets.assign(row_offsets, row_offsets + K + 1);
  alloc(comp, comp->offsets, (K + 1) * sizeof(int64_t));
  alloc(comp, comp->A, (size_t)N * R * 4);
  alloc(comp, comp->Bk, (size_t)K * R * 4);
  comp->Jq = round_up(J, 64);
  alloc(comp, comp->M, (size_t)3 * K * R * comp->Jq * 2);
  alloc(comp, comp->D, (size_t)J * R * 4);
  alloc(comp, comp->E, (size_t)R * 4);
  alloc(comp, comp->Ft, (size_t)K * R * R * 4);
  alloc(comp, comp->xnorm2, (size_t)K * 8);
  alloc(comp, comp->rank1, (size_t)K * 4);
  alloc(comp, comp->DtD, (size_t)R * R * 8);
  h2d_i64(ctx, static_cast<int64_t*>(comp->offsets.p), row_offsets, (K + 1), s);
  return comp;
}

// The stage-1 test matrix (Alg. 1: the caller's, or the Gaussian stream
// (seed, 0) rounded to bf16-representable values), padded to Jpad x LP and
// rounded to X's 16-bit type.
const float* prepare_omega(dpar2_ctx* ctx, int J, int ell, int LP, dpar2_dtype dtype, const dpar2_options* opt,
                           const float* omega, cudaStream_t s) {
  const int Jpad = round_up(J, 32);
  const float* om = omega;
  if (!om) {
    float* g = wsget<float>(ctx, "omega", (size_t)J * ell);
    launch_gaussian(opt->seed, 0, (int64_t)J * ell, g, 1, s);
    om = g;
  }
  float* om_pad = wsget<float>(ctx, "om_pad", (size_t)Jpad * LP);
  launch_pad_omega(om, J, ell, Jpad, LP, dtype, om_pad, s);
  return om_pad;
}

}  // namespace

// ------------------------------------------------------------ ctx / comp ----
void* dpar2_ctx::get(const std::string& name, size_t bytes) {
  auto& b = ws[name];
  if (b.p && b.bytes >= bytes) return b.p;
  if (b.p) {
    cudaDeviceSynchronize();
    cudaFree(b.p);
  }
  b.p = nullptr;
  b.bytes = 0;
  const size_t want = std::max<size_t>(bytes, 256);
  if (cudaMalloc(&b.p, want) != cudaSuccess) {
    cudaGetLastError();
    b.p = nullptr;
    return nullptr;
  }
  b.bytes = want;
  return b.p;
}

size_t dpar2_comp::device_bytes() const {
  return offsets.bytes + A.bytes + Bk.bytes + M.bytes + D.bytes + E.bytes + Ft.bytes + xnorm2.bytes + rank1.bytes +
         DtD.bytes;
}

dpar2_comp::~dpar2_comp() {
  for (dp2::DevBuf* b : {&offsets, &A, &Bk, &M, &D, &E, &Ft, &xnorm2, &rank1, &DtD}) release(this, *b);
}

extern "C" {

dpar2_status dpar2_options_default(dpar2_options* opt) {
  if (!opt) return DPAR2_ERR_INVALID_ARG;
  opt->R = 10;
  opt->p = 10;
  opt->q = 0;
  opt->seed = 0;
  opt->max_iter = 32;
  opt->tol = -1.0;
  opt->schedule = -1;
  opt->flags = 0;
  opt->proj_cols = 0;
  return DPAR2_OK;
}

dpar2_status dpar2_create(dpar2_ctx** out, int device) {
  if (!out) return DPAR2_ERR_INVALID_ARG;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
    cudaGetLastError();
    return DPAR2_ERR_CUDA;
  }
  int prev = -1;
  cudaGetDevice(&prev);
  if (cudaSetDevice(device) != cudaSuccess) return DPAR2_ERR_CUDA;
  dpar2_ctx* ctx = new dpar2_ctx();
  ctx->device = device;
  cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
  cudaStream_t work;
  cudaEvent_t ev;
  if (cudaMalloc(&ctx->d_status, sizeof(int)) != cudaSuccess ||
      cudaMallocHost(&ctx->h_status, 64) != cudaSuccess ||  // status word + pinned scalars
      cudaStreamCreateWithFlags(&work, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    delete ctx;
    if (prev >= 0) cudaSetDevice(prev);
    return DPAR2_ERR_CUDA;
  }
  for (int i = 0; i < 2 * DPAR2_NUM_PHASES; ++i) cudaEventCreate(&ctx->tev[i]);
  cudaMemPoolProps pp = {};
  pp.allocType = cudaMemAllocationTypePinned;
  pp.handleTypes = cudaMemHandleTypeNone;
  pp.location.type = cudaMemLocationTypeDevice;
  pp.location.id = device;
  if (cudaMemPoolCreate(&ctx->pool, &pp) == cudaSuccess) {
    uint64_t keep = UINT64_MAX;  // freed buffers stay in the pool for the next objects
    cudaMemPoolSetAttribute(ctx->pool, cudaMemPoolAttrReleaseThreshold, &keep);
  } else {
    cudaGetLastError();
    ctx->pool = nullptr;
  }
  ctx->ws["__work_stream"].p = reinterpret_cast<void*>(work);
  ctx->ws["__event"].p = reinterpret_cast<void*>(ev);
  *out = ctx;
  if (prev >= 0) cudaSetDevice(prev);
  return DPAR2_OK;
}

void dpar2_destroy(dpar2_ctx* ctx) {
  if (!ctx || ctx->closing) return;
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(ctx->device);
  ctx_release(ctx);
  if (prev >= 0) cudaSetDevice(prev);
}

const char* dpar2_last_error(const dpar2_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }
long long dpar2_kernel_launches(void) { return g_launches.load(); }
int dpar2_last_info(const dpar2_ctx* ctx) {
  return (ctx && ctx->h_status) ? (*ctx->h_status & (ST_RANK_DROP | ST_SWEEP_CAP | ST_PINV)) : 0;
}

dpar2_status dpar2_upload_rows(dpar2_ctx* ctx, const void* Xh, int64_t rows, int J, dpar2_dtype dtype, void* Xd,
                               int64_t ldx, void* stream) {
  if (!ctx) return DPAR2_ERR_INVALID_ARG;
  if (!Xh || !Xd || rows < 0 || J < 1 || ldx < J) {
    ctx->err = "dpar2_upload_rows: null buffer or ldx < J";
    return DPAR2_ERR_INVALID_ARG;
  }
  const size_t es = dtype_size(dtype);
  return guarded(ctx, stream, [&](cudaStream_t s) {
    if (rows == 0) return;
    const size_t rowb = (size_t)J * es;
    if (ldx == J) {
      CK(cudaMemcpyAsync(Xd, Xh, (size_t)rows * rowb, cudaMemcpyHostToDevice, s));
      return;
    }
    // Packed rows -> pitched rows: contiguous copies of ~128 MB chunks into four
    // device staging buffers, alternating between two copy streams (two copy
    // engines in flight), each chunk re-pitched on the work stream by a kernel
    // (a 2-D copy of short rows moves far below the link's bandwidth).  Chunk
    // c + 4 waits for the kernel that read buffer c % 4.
    constexpr int NB = 4, NCS = 2;
    const int64_t crow = std::max<int64_t>(1, (int64_t)((128u << 20) / rowb));
    uint8_t* stage = wsget<uint8_t>(ctx, "up_stage", NB * (size_t)crow * rowb);
    cudaStream_t cs[NCS];
    for (int i = 0; i < NCS; ++i) {
      auto& e = ctx->ws[std::string("__copy_stream") + char('0' + i)];
      if (!e.p) {
        cudaStream_t x;
        CK(cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking));
        e.p = reinterpret_cast<void*>(x);
      }
      cs[i] = reinterpret_cast<cudaStream_t>(e.p);
    }
    cudaEvent_t ev[2 * NB + 1];  // copied[b], used[b], start
    for (int i = 0; i < 2 * NB + 1; ++i) {
      auto& e = ctx->ws[std::string("__copy_ev") + char('a' + i)];
      if (!e.p) {
        cudaEvent_t x;
        CK(cudaEventCreateWithFlags(&x, cudaEventDisableTiming));
        e.p = reinterpret_cast<void*>(x);
      }
      ev[i] = reinterpret_cast<cudaEvent_t>(e.p);
    }
    CK(cudaEventRecord(ev[2 * NB], s));  // the copies start after the work stream's prior work
    for (int i = 0; i < NCS; ++i) CK(cudaStreamWaitEvent(cs[i], ev[2 * NB], 0));
    int64_t c = 0;
    for (int64_t r0 = 0; r0 < rows; r0 += crow, ++c) {
      const int b = (int)(c % NB);
      cudaStream_t q = cs[c % NCS];
      const int64_t nr = std::min<int64_t>(crow, rows - r0);
      if (c >= NB) CK(cudaStreamWaitEvent(q, ev[NB + b], 0));  // kernel done with buffer b
      CK(cudaMemcpyAsync(stage + (size_t)b * crow * rowb, static_cast<const uint8_t*>(Xh) + (size_t)r0 * rowb,
                         (size_t)nr * rowb, cudaMemcpyHostToDevice, q));
      CK(cudaEventRecord(ev[b], q));
      CK(cudaStreamWaitEvent(s, ev[b], 0));
      launch_repitch(stage + (size_t)b * crow * rowb, nr, J, (int)es, static_cast<uint8_t*>(Xd) + (size_t)r0 * ldx * es,
                     ldx, s);
      CK(cudaEventRecord(ev[NB + b], s));
    }
  });
}

dpar2_status dpar2_scratch(dpar2_ctx* ctx, const char* name, void** ptr, size_t* bytes) {
  if (!ctx || !name || !ptr || !bytes) return DPAR2_ERR_INVALID_ARG;
  auto it = ctx->ws.find(name);
  if (it == ctx->ws.end() || name[0] == '_' || !it->second.p) {
    ctx->err = std::string("no scratch buffer named ") + name;
    return DPAR2_ERR_INVALID_ARG;
  }
  *ptr = it->second.p;
  *bytes = it->second.bytes;
  return DPAR2_OK;
}

dpar2_status dpar2_set_timing(dpar2_ctx* ctx, int enable) {
  if (!ctx) return DPAR2_ERR_INVALID_ARG;
  ctx->timing = enable != 0;
  return DPAR2_OK;
}

int dpar2_last_timings(const dpar2_ctx* ctx, double* ms, int n) {
  if (!ctx || !ms) return 0;
  const int m = std::min(n, (int)DPAR2_NUM_PHASES);
  for (int i = 0; i < m; ++i) ms[i] = ctx->tms[i];
  return m;
}

dpar2_status dpar2_gaussian(dpar2_ctx* ctx, uint64_t seed, uint32_t stream_id, int64_t n, float* out, int round16,
                            void* stream) {
  if (!ctx) return DPAR2_ERR_INVALID_ARG;
  if (!out || n < 0) {
    ctx->err = "dpar2_gaussian: out is null or n < 0";
    return DPAR2_ERR_INVALID_ARG;
  }
  return guarded(ctx, stream, [&](cudaStream_t s) {
    if (n > 0) launch_gaussian(seed, stream_id, n, out, round16, s);
  });
}

dpar2_status dpar2_philox_words(dpar2_ctx* ctx, uint64_t seed, uint32_t stream_id, int64_t n, uint32_t* out,
                                void* stream) {
  if (!ctx) return DPAR2_ERR_INVALID_ARG;
  if (!out || n < 0) {
    ctx->err = "dpar2_philox_words: out is null or n < 0";
    return DPAR2_ERR_INVALID_ARG;
  }
  return guarded(ctx, stream, [&](cudaStream_t s) {
    if (n > 0) launch_philox_words(seed, stream_id, n, out, s);
  });
}

// --------------------------------------------------------------- compress ----
dpar2_status dpar2_compress(dpar2_ctx* ctx, int K, int J, const int64_t* row_offsets, const void* X, int64_t ldx,
                            dpar2_dtype dtype, const dpar2_options* opt, const float* omega, const float* omega2,
                            dpar2_comp** out, void* stream) {
  if (!ctx) return DPAR2_ERR_INVALID_ARG;
  dpar2_status st0 = check_compress(ctx, K, J, row_offsets, X, ldx, dtype, opt, out, true);
  if (st0 != DPAR2_OK) return st0;
  dpar2_comp* comp = nullptr;
  dpar2_status st = guarded(ctx, stream, [&](cudaStream_t s) {
    comp = new_comp(ctx, K, J, row_offsets, opt, s);
    tbegin(ctx, s, DPAR2_PH_COMPRESS);
    const float* om_pad = prepare_omega(ctx, J, comp->ell, comp->LP, dtype, opt, omega, s);
    // ---- stage 1 over all slices ----
    stage1_range(ctx, comp, X, ldx, dtype, opt, 0, K, row_offsets, static_cast<const int64_t*>(comp->offsets.p),
                 om_pad, true, s);
    // ---- stage 2: randomized SVD of M (J x KR) ----
    stage2_all(ctx, comp, opt, omega2, s);
    tend(ctx, s, DPAR2_PH_COMPRESS);
    if (opt->flags & DPAR2_FLAG_DROP_M) {
      alloc(comp, comp->M, 0);  // stream-ordered after the kernels that read it
    }
  });
  if (st != DPAR2_OK) {
    if (comp) dpar2_comp_free(comp);
    return st;
  }
  *out = comp;
  return DPAR2_OK;
}

// ------------------------------------------------- compress from host memory ----
// Chunks of whole slices are copied host -> device on a copy stream, each
// into its own staging buffer (two in turn); the work stream re-pitches a
// chunk into its device rows and runs stage 1 on it while the next chunk
// copies, so X crosses the host link once and the transfers hide the stage-1
// work.  Stage 2 and everything after it need only the compressed factors.
dpar2_status dpar2_compress_host(dpar2_ctx* ctx, int K, int J, const int64_t* row_offsets, const void* X_host,
                                 dpar2_dtype dtype, const dpar2_options* opt, const float* omega,
                                 const float* omega2, void* X_dev, int64_t ldx, size_t chunk_bytes,
                                 dpar2_comp** out, void* stream) {
  if (!ctx) return DPAR2_ERR_INVALID_ARG;
  const size_t es = (dtype == DPAR2_F32) ? 4 : 2;
  // device row pitch: the caller's, or rows padded to 32 bytes in the chunk buffers
  const int64_t ldd = X_dev ? ldx : (int64_t)((J * es + 31) / 32 * 32 / es);
  dpar2_status st0 = check_compress(ctx, K, J, row_offsets, X_dev ? X_dev : X_host, ldd, dtype, opt, out, X_dev != nullptr);
  if (st0 != DPAR2_OK) return st0;
  if (!X_host) {
    ctx->err = "X_host must be non-null";
    return DPAR2_ERR_INVALID_ARG;
  }
  dpar2_comp* comp = nullptr;
  dpar2_status st = guarded(ctx, stream, [&](cudaStream_t s) {
    comp = new_comp(ctx, K, J, row_offsets, opt, s);
    tbegin(ctx, s, DPAR2_PH_COMPRESS);
    const float* om_pad = prepare_omega(ctx, J, comp->ell, comp->LP, dtype, opt, omega, s);
    // chunks of whole slices, about chunk_bytes of X each
    const size_t rowb = (size_t)J * es;
    // 2 GB by default: the per-chunk latency of the small stage-1 kernels shows
    // in the total (1 GB: 77.6 ms, 2 GB: 75.4 ms, 4 GB: 75.1 ms for the 13.2 GB
    // spectrogram tensor over a 211 GB/s link, whose copy alone takes 62.5 ms)
    const size_t target = chunk_bytes ? chunk_bytes : ((size_t)2 << 30);
    std::vector<int> cut{0};
    for (int k = 0; k < K; ++k) {
      const int64_t rows = row_offsets[k + 1] - row_offsets[cut.back()];
      if (k + 1 < K && (size_t)rows * rowb >= target) cut.push_back(k + 1);
    }
    cut.push_back(K);
    const int nc = (int)cut.size() - 1;
    int64_t maxrows = 0;
    for (int c = 0; c < nc; ++c) maxrows = std::max(maxrows, row_offsets[cut[c + 1]] - row_offsets[cut[c]]);
    // NB landing buffers: the copy of chunk c + NB is queued right after the
    // work stream's use of chunk c's buffer, so the copy engine runs up to NB
    // chunks ahead of the host's stage-1 launches
    constexpr int NB = 3;
    const bool direct = ldd == J;  // host rows already have the device pitch: no staging
    uint8_t* stage = direct ? nullptr : wsget<uint8_t>(ctx, "hc_stage", (size_t)NB * maxrows * rowb);
    uint8_t* cbuf = X_dev ? nullptr : wsget<uint8_t>(ctx, "hc_chunk", (size_t)NB * maxrows * ldd * es);
    int64_t* d_coff = wsget<int64_t>(ctx, "hc_off", (size_t)NB * (K + 1));
    auto& cse = ctx->ws["__copy_stream0"];
    if (!cse.p) {
      cudaStream_t x;
      CK(cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking));
      cse.p = reinterpret_cast<void*>(x);
    }
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(cse.p);
    cudaEvent_t ev[2 * NB + 1];  // copied[b], free[b], start
    for (int i = 0; i < 2 * NB + 1; ++i) {
      auto& e = ctx->ws[std::string("__copy_ev") + char('a' + i)];
      if (!e.p) {
        cudaEvent_t x;
        CK(cudaEventCreateWithFlags(&x, cudaEventDisableTiming));
        e.p = reinterpret_cast<void*>(x);
      }
      ev[i] = reinterpret_cast<cudaEvent_t>(e.p);
    }
    auto dst_of = [&](int c) -> uint8_t* {
      const int64_t r0 = row_offsets[cut[c]];
      return X_dev ? static_cast<uint8_t*>(X_dev) + (size_t)r0 * ldd * es : cbuf + (size_t)(c % NB) * maxrows * ldd * es;
    };
    auto land_of = [&](int c) -> uint8_t* { return direct ? dst_of(c) : stage + (size_t)(c % NB) * maxrows * rowb; };
    auto queue_copy = [&](int c) {
      const int b = c % NB;
      const int64_t r0 = row_offsets[cut[c]], nr = row_offsets[cut[c + 1]] - r0;
      // the landing buffer is free once the work stream re-pitched (staging) or
      // compressed (direct into a chunk buffer) chunk c - NB
      if (c >= NB) CK(cudaStreamWaitEvent(cs, ev[NB + b], 0));
      CK(cudaMemcpyAsync(land_of(c), static_cast<const uint8_t*>(X_host) + (size_t)r0 * rowb, (size_t)nr * rowb,
                         cudaMemcpyHostToDevice, cs));
      CK(cudaEventRecord(ev[b], cs));
    };
    CK(cudaEventRecord(ev[2 * NB], s));  // copies start after the work stream's prior work
    CK(cudaStreamWaitEvent(cs, ev[2 * NB], 0));
    for (int c = 0; c < std::min(NB, nc); ++c) queue_copy(c);
    std::vector<int64_t> loc;
    for (int c = 0; c < nc; ++c) {
      const int b = c % NB, k0 = cut[c], Kc = cut[c + 1] - cut[c];
      const int64_t r0 = row_offsets[k0], nr = row_offsets[cut[c + 1]] - r0;
      uint8_t* dst = dst_of(c);
      CK(cudaStreamWaitEvent(s, ev[b], 0));
      if (!direct) {
        launch_repitch(land_of(c), nr, J, (int)es, dst, ldd, s);
        CK(cudaEventRecord(ev[NB + b], s));
        if (c + NB < nc) queue_copy(c + NB);
      }
      loc.assign(Kc + 1, 0);
      for (int k = 0; k <= Kc; ++k) loc[k] = row_offsets[k0 + k] - r0;
      int64_t* d_loc = d_coff + (size_t)b * (K + 1);
      h2d_i64(ctx, d_loc, loc.data(), Kc + 1, s);
      stage1_range(ctx, comp, dst, ldd, dtype, opt, k0, Kc, loc.data(), d_loc, om_pad, false, s);
      if (direct) {
        CK(cudaEventRecord(ev[NB + b], s));
        if (c + NB < nc) queue_copy(c + NB);
      }
    }
    stage2_all(ctx, comp, opt, omega2, s);
    tend(ctx, s, DPAR2_PH_COMPRESS);
    if (opt->flags & DPAR2_FLAG_DROP_M) alloc(comp, comp->M, 0);
  });
  if (st != DPAR2_OK) {
    if (comp) dpar2_comp_free(comp);
    return st;
  }
  *out = comp;
  return DPAR2_OK;
}

// -------------------------------------------------------------------- fit ----
dpar2_status dpar2_fit(dpar2_ctx* ctx, const dpar2_comp* comp, const dpar2_options* opt, const float* V0, float* H,
                       float* V, float* W, float* Upol, float* U, double* loss_history, int* iters_run,
                       double* fitness, void* stream) {
  if (!ctx) return DPAR2_ERR_INVALID_ARG;
  if (!comp || !opt || !H || !V || !W) {
    ctx->err = "comp, opt, H, V and W must be non-null";
    return DPAR2_ERR_INVALID_ARG;
  }
  if (opt->R != comp->R || opt->max_iter < 1) {
    ctx->err = "opt->R must equal the compression's R and max_iter >= 1";
    return DPAR2_ERR_SHAPE;
  }
  if (fitness && !comp->M.p) {
    ctx->err = "fitness needs M (compressed without DPAR2_FLAG_DROP_M)";
    return DPAR2_ERR_INVALID_ARG;
  }
  int iters = 0;
  double fit_val = 0.0;
  std::vector<double> hist(opt->max_iter, 0.0);
  dpar2_status st = guarded(ctx, stream, [&](cudaStream_t s) {
    const int K = comp->K, J = comp->J, R = comp->R, RR = R * R;
    const float* v0 = V0;
    if (!v0) {
      float* g = wsget<float>(ctx, "V0", (size_t)J * R);
      launch_gaussian(opt->seed, 3, (int64_t)J * R, g, 0, s);
      v0 = g;
    }
    AlsBufs b;
    b.K = K;
    b.J = J;
    b.R = R;
    b.D = static_cast<const float*>(comp->D.p);
    b.Ft = static_cast<const float*>(comp->Ft.p);
    b.DtD = static_cast<const double*>(comp->DtD.p);
    b.H = H;
    b.W = W;
    b.CV = wsget<float>(ctx, "CV", RR);
    b.Upol = Upol ? Upol : wsget<float>(ctx, "Upol", (size_t)K * RR);
    b.Pi = wsget<float>(ctx, "Pi", (size_t)K * RR);
    b.Prot = (opt->flags & DPAR2_FLAG_COLD_QSTEP) ? nullptr : wsget<float>(ctx, "Prot", (size_t)K * RR);
    b.rank = static_cast<const int*>(comp->rank1.p);
    double* d6 = wsget<double>(ctx, "als_d", (size_t)7 * RR);
    b.Psi = d6;
    b.VtV = d6 + RR;
    b.HtH = d6 + 2 * RR;
    b.WtW = d6 + 3 * RR;
    b.Ginv = d6 + 4 * RR;
    b.InvH = d6 + 5 * RR;
    b.InvV = d6 + 6 * RR;
    const bool three = als3_supported(R) && !(opt->flags & DPAR2_FLAG_FIVE_LAUNCH);
    b.nblk = three ? als3_blocks(K, R, ctx->num_sms) : als_blocks(K, R, ctx->num_sms);
    b.nq = qstep_blocks(K, R, b.nblk);
    b.pr = std::max(b.nblk, b.nq);
    b.part = wsget<float>(ctx, "als_part", (size_t)3 * b.pr * (2 * RR + 2));
    b.loss = wsget<double>(ctx, "als_loss", (size_t)opt->max_iter);
    b.small = wsget<double>(ctx, "als_small", (size_t)8 * RR + 8);
    b.atb = wsget<float>(ctx, "atb_part", (size_t)kAtbBlocks * RR);
    b.status = ctx->d_status;
    auto iterate = [&](int it) {
      if (three) launch_als_iteration3(b, it, s);
      else launch_als_iteration(b, it, s);
    };
    tbegin(ctx, s, DPAR2_PH_ALS);
    // one persistent launch for the whole loop (fixed iteration count, R <= 20,
    // every slice in one pass of the slice blocks' warps)
    bool persisted = false;
    if (opt->tol < 0 && persist_supported(R) && ctx->num_sms >= 2 && K <= persist_capacity(R, ctx->num_sms) &&
        !(opt->flags & (DPAR2_FLAG_FIVE_LAUNCH | DPAR2_FLAG_NO_PERSIST))) {
      const int nsb = ctx->num_sms - 1;
      AlsBufs bp = b;
      bp.nblk = bp.nq = bp.pr = nsb;
      bp.pstride = round_up(2 * RR + 2, 4);
      bp.part = wsget<float>(ctx, "als_part_p", (size_t)3 * nsb * bp.pstride);
      PersistArgs pa;
      pa.K = K;
      pa.R = R;
      pa.max_iter = opt->max_iter;
      pa.pstride = bp.pstride;
      pa.wstride = 0;
      pa.Ft = b.Ft;
      pa.DtD = b.DtD;
      pa.rank = b.rank;
      pa.H = b.H;
      pa.W = b.W;
      pa.CV = b.CV;
      pa.Upol = b.Upol;
      pa.Pi = b.Pi;
      pa.Prot = b.Prot;
      pa.Psi = b.Psi;
      pa.VtV = b.VtV;
      pa.HtH = b.HtH;
      pa.WtW = b.WtW;
      pa.Ginv = b.Ginv;
      pa.InvH = b.InvH;
      pa.InvV = b.InvV;
      pa.part1 = bp.part;
      pa.part2 = bp.part + (size_t)nsb * pa.pstride;
      pa.part3 = bp.part + (size_t)2 * nsb * pa.pstride;
      pa.loss = b.loss;
      pa.status = b.status;
      pa.bar = wsget<unsigned>(ctx, "als_bar", 4);
      pa.abort = nullptr;
      launch_als_init(bp, v0, s);
      if (launch_als_persist(pa, ctx->num_sms, s)) {
        launch_als_finish(bp, opt->max_iter - 1, s);
        b = bp;
        persisted = true;
        iters = opt->max_iter;
      }
    }
    if (!persisted) launch_als_init(b, v0, s);
    if (!persisted && opt->tol < 0) {
      bool graph = !(opt->flags & DPAR2_FLAG_NO_GRAPH);
      if (graph) {
        cudaGraph_t g;
        cudaGraphExec_t ge;
        const long long c0 = g_launches.load();
        CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        for (int it = 0; it < opt->max_iter; ++it) iterate(it);
        launch_als_finish(b, opt->max_iter - 1, s);
        CK(cudaStreamEndCapture(s, &g));
        const long long captured = g_launches.load() - c0;
        g_launches.fetch_sub(captured);
        CK(cudaGraphInstantiate(&ge, g, 0));
        CK(cudaGraphLaunch(ge, s));
        g_launches.fetch_add(captured);
        cudaGraphExecDestroy(ge);  // freed when the launch completes
        cudaGraphDestroy(g);
      } else {
        for (int it = 0; it < opt->max_iter; ++it) iterate(it);
        launch_als_finish(b, opt->max_iter - 1, s);
      }
      iters = opt->max_iter;
    } else if (!persisted) {
      double prev = 0.0;
      for (int it = 0; it < opt->max_iter; ++it) {
        iterate(it);
        launch_als_finish(b, it, s);
        double e = 0.0;
        CK(cudaMemcpyAsync(&e, b.loss + it, sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        iters = it + 1;
        if (it > 0 && prev - e <= opt->tol * prev) break;
        prev = e;
      }
    }
    tend(ctx, s, DPAR2_PH_ALS);
    tbegin(ctx, s, DPAR2_PH_OUTPUT);
    // outputs: V = D CV (Lemma 2 keeps V in span(D)), U_k = A_k Upol_k H
    int64_t* off2 = wsget<int64_t>(ctx, "off_fit", 2);
    const int64_t h2[2] = {0, (int64_t)J};
    h2d_i64(ctx, off2, h2, sizeof(h2) / sizeof(int64_t), s);
    launch_seg_product(b.D, R, R, b.CV, 0, R, V, R, off2, 1, J, s);
    if (U) {
      float* Tk = wsget<float>(ctx, "Tk", (size_t)K * RR);
      launch_upol_h(K, R, b.Upol, H, Tk, s);
      launch_seg_product(static_cast<const float*>(comp->A.p), R, R, Tk, RR, R, U, R,
                         static_cast<const int64_t*>(comp->offsets.p), K, comp->maxI, s);
    }
    if (loss_history) CK(cudaMemcpyAsync(hist.data(), b.loss, iters * sizeof(double), cudaMemcpyDeviceToHost, s));
    if (fitness) {
      float* P = wsget<float>(ctx, "Pk", (size_t)K * RR);
      double* fpart = wsget<double>(ctx, "fit_part", (size_t)b.nblk + 4);
      launch_p_from_cv(K, R, b.CV, b.Ft, P, s);
      launch_fitness(K, R, P, b.Upol, H, W, b.VtV, static_cast<const double*>(comp->xnorm2.p), fpart, b.nblk,
                     fpart + b.nblk, s);
      DP2_COUNTED(k_sum_f64<<<1, 256, 0, s>>>(static_cast<const double*>(comp->xnorm2.p), K, fpart + b.nblk + 1));
      tend(ctx, s, DPAR2_PH_OUTPUT);
      double h[2];
      CK(cudaMemcpyAsync(h, fpart + b.nblk, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      fit_val = h[1] > 0 ? 1.0 - h[0] / h[1] : 0.0;
    } else {
      tend(ctx, s, DPAR2_PH_OUTPUT);
    }
  });
  if (st == DPAR2_OK) {
    if (loss_history) std::copy(hist.begin(), hist.begin() + iters, loss_history);
    if (iters_run) *iters_run = iters;
    if (fitness) *fitness = fit_val;
  }
  return st;
}

// ------------------------------------------------------ reconstruct error ----
dpar2_status dpar2_reconstruct_error(dpar2_ctx* ctx, const dpar2_comp* comp, const void* X, int64_t ldx,
                                     dpar2_dtype dtype, const float* H, const float* V, const float* W,
                                     const float* Upol, double* sq_err, double* fitness, void* stream) {
  if (!ctx) return DPAR2_ERR_INVALID_ARG;
  if (!comp || !H || !V || !W) {
    ctx->err = "comp, H, V and W must be non-null";
    return DPAR2_ERR_INVALID_ARG;
  }
  if (X) {
    try {
      require(dtype == DPAR2_F32 || dtype == DPAR2_BF16 || dtype == DPAR2_F16, DPAR2_ERR_INVALID_ARG, "bad dtype");
      require(ldx >= comp->J, DPAR2_ERR_SHAPE, "ldx < J");
      require((ldx * (int64_t)dtype_size(dtype)) % 16 == 0, DPAR2_ERR_INVALID_ARG,
              "ldx * sizeof(dtype) must be a multiple of 16 bytes");
      require((reinterpret_cast<uintptr_t>(X) & 15) == 0, DPAR2_ERR_INVALID_ARG, "X must be 16-byte aligned");
    } catch (const Fail& f) {
      ctx->err = f.msg;
      return f.st;
    }
  } else if (!comp->M.p) {
    ctx->err = "identity mode needs M (compressed without DPAR2_FLAG_DROP_M)";
    return DPAR2_ERR_INVALID_ARG;
  }
  double res[2] = {0, 0};
  dpar2_status st = guarded(ctx, stream, [&](cudaStream_t s) {
    const int K = comp->K, J = comp->J, R = comp->R, RR = R * R;
    double* d6 = wsget<double>(ctx, "re_d", (size_t)6 * RR);
    double* Psi = d6;
    double* VtV = d6 + RR;
    launch_psi_vtv(J, R, static_cast<const float*>(comp->D.p), V, Psi, VtV,
                   wsget<float>(ctx, "atb_part", (size_t)kAtbBlocks * RR), s);
    const int nblk = als_blocks(K, R, ctx->num_sms);
    const float* up = Upol;
    if (!up) {
      AlsBufs b;
      b.K = K;
      b.J = J;
      b.R = R;
      b.D = static_cast<const float*>(comp->D.p);
      b.Ft = static_cast<const float*>(comp->Ft.p);
      b.H = const_cast<float*>(H);
      b.W = const_cast<float*>(W);
      b.Psi = Psi;
      b.Upol = wsget<float>(ctx, "re_upol", (size_t)K * RR);
      b.Pi = wsget<float>(ctx, "re_pi", (size_t)K * RR);
      b.nq = qstep_blocks(K, R, nblk);
      b.rank = static_cast<const int*>(comp->rank1.p);
      b.pr = std::max(nblk, b.nq);
      b.part = wsget<float>(ctx, "re_part", (size_t)3 * b.pr * (2 * RR + 2));
      b.status = ctx->d_status;
      b.nblk = nblk;
      launch_qstep_only(b, s);
      up = b.Upol;
    }
    float* P = wsget<float>(ctx, "re_P", (size_t)K * RR);
    double* fpart = wsget<double>(ctx, "re_fit", (size_t)nblk + 4);
    if (!X) {
      // identity mode: A_k^T X_k = B_k C_k^T, so V^T M_k stands for V^T X_k^T A_k
      launch_vtm(K, J, R, V, comp->M.p, (int64_t)K * R * comp->Jq, comp->Jq, P, s);
      launch_fitness(K, R, P, up, H, W, VtV, static_cast<const double*>(comp->xnorm2.p), fpart, nblk, fpart + nblk,
                     s);
      DP2_COUNTED(k_sum_f64<<<1, 256, 0, s>>>(static_cast<const double*>(comp->xnorm2.p), K, fpart + nblk + 1));
    } else {
      // streamed mode: one pass over X projects it onto A_k (A_k^T X_k and
      // ||X_k||^2 measured, not taken from the compression) and A_k^T A_k is
      // formed, so the error assumes neither the stage-1 identity nor A_k's
      // orthonormality
      const int LP = round_up(R, 8), Jp = round_up(J, 4), LPN = tc_lpn(R);
      const int64_t N = comp->N;
      const int64_t* d_off = static_cast<const int64_t*>(comp->offsets.p);
      float* Ap = wsget<float>(ctx, "re_Ap", (size_t)N * LP);
      launch_pad_omega(static_cast<const float*>(comp->A.p), (int)N, R, (int)N, LP, DPAR2_F32, Ap, s);
      double* G = wsget<double>(ctx, "re_AtA", (size_t)K * LP * LP);
      const int nsplit = gram_splits(K, comp->maxI);
      double* Gp = nsplit > 1 ? wsget<double>(ctx, "re_AtAp", (size_t)K * nsplit * LP * LP) : nullptr;
      launch_gram_dd(Ap, LP, d_off, K, R, G, Gp, nsplit, s);
      float* Bs = wsget<float>(ctx, "re_B", (size_t)K * LP * Jp);
      double* xn = wsget<double>(ctx, "re_xn", (size_t)K);
      bool projected = false;
      if (dtype != DPAR2_F32 && tc_available()) {
        std::vector<int64_t> hp(K + 1, 0);
        int64_t maxPad = 0;
        for (int k = 0; k < K; ++k) {
          const int64_t pk = round_up64(comp->h_offsets[k + 1] - comp->h_offsets[k], 64);
          hp[k + 1] = hp[k] + pk;
          maxPad = std::max(maxPad, pk);
        }
        int64_t* d_poff = wsget<int64_t>(ctx, "re_poff", (size_t)K + 1);
        h2d_i64(ctx, d_poff, hp.data(), (K + 1), s);
        int PNS = 0, POFF = 0;
        proj_layout(R, &PNS, &POFF);
        void* Qs = wsget<uint16_t>(ctx, "re_Qs", (size_t)PNS * hp[K]);
        launch_qsplit(Ap, LP, PNS, POFF, d_off, d_poff, K, hp[K], maxPad, dtype, Qs, s);
        const int nJb = (Jp + project_tc_cols(PNS) - 1) / project_tc_cols(PNS);
        double* xp = wsget<double>(ctx, "re_xpart_tc", (size_t)K * nJb * kProjNormWarps);
        projected = launch_project_tc(X, dtype, ldx, N, d_off, d_poff, K, J, Jp, Qs, hp[K], PNS, POFF, LP, Bs, xp, nJb,
                                      true, ctx->num_sms, ctx->d_status, s);
        if (projected) launch_reduce_rows_f64(xp, K, nJb * kProjNormWarps, xn, s);
      }
      if (!projected) {
        const int nJb = project_blocks(Jp, LP);
        double* xp = wsget<double>(ctx, "re_xpart", (size_t)K * nJb);
        launch_project_generic(X, dtype, ldx, d_off, K, J, Jp, Ap, LP, Bs, xp, nullptr, s);
        launch_reduce_rows_f64(xp, K, nJb, xn, s);
      }
      launch_p_stream(K, J, Jp, R, LP, V, Bs, P, s);
      launch_fitness(K, R, P, up, H, W, VtV, xn, fpart, nblk, fpart + nblk, s, G, LP);
      DP2_COUNTED(k_sum_f64<<<1, 256, 0, s>>>(xn, K, fpart + nblk + 1));
    }
    CK(cudaMemcpyAsync(res, fpart + nblk, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
  });
  if (st == DPAR2_OK) {
    if (sq_err) *sq_err = res[0];
    if (fitness) *fitness = res[1] > 0 ? 1.0 - res[0] / res[1] : 0.0;
  }
  return st;
}

// ------------------------------------- reconstruct error without allocation ----
// Some callers must not allocate device memory inside a call: a serving loop
// that reserves all of its device memory up front in its own pool, or one that
// cannot take the device-wide synchronisation of a cudaFree when the
// context's grow-only scratch has to grow for a larger problem.  For them the
// identity-mode error evaluation has a variant whose scratch is a fixed array
// in the library's device image (one per device, created when the module is
// loaded), carved into its buffers on every call.
static __device__ __align__(256) unsigned char g_noalloc_scratch[DPAR2_NOALLOC_SCRATCH_BYTES];

namespace {
// Device address of the array in the current device's context.  Looked up on
// every call (cudaGetSymbolAddress allocates nothing) rather than cached, so a
// context that was reset and re-created since the last call gets the address
// of its own copy of the array.
void* noalloc_base() {
  void* p = nullptr;
  CK(cudaGetSymbolAddress(&p, g_noalloc_scratch));
  require(p != nullptr, DPAR2_ERR_CUDA, "cudaGetSymbolAddress returned a null address");
  return p;
}

size_t up256(size_t b) { return (b + 255) / 256 * 256; }
}  // namespace

dpar2_status dpar2_reconstruct_error_noalloc(dpar2_ctx* ctx, const dpar2_comp* comp, const float* H, const float* V,
                                             const float* W, const float* Upol, double* sq_err, double* fitness,
                                             void* stream) {
  if (!ctx) return DPAR2_ERR_INVALID_ARG;
  if (!comp || !H || !V || !W || !Upol) {
    ctx->err = "comp, H, V, W and Upol must be non-null";
    return DPAR2_ERR_INVALID_ARG;
  }
  if (!comp->M.p) {
    ctx->err = "identity mode needs M (compressed without DPAR2_FLAG_DROP_M)";
    return DPAR2_ERR_INVALID_ARG;
  }
  const int K = comp->K, J = comp->J, R = comp->R, RR = R * R;
  const int nblk = als_blocks(K, R, ctx->num_sms);
  // P_k = V^T M_k, Psi and V^T V, the A^T B block partials, the fitness partials
  const size_t bP = up256((size_t)K * RR * sizeof(float));
  const size_t bD = up256((size_t)2 * RR * sizeof(double));
  const size_t bA = up256((size_t)kAtbBlocks * RR * sizeof(float));
  const size_t bF = up256(((size_t)nblk + 4) * sizeof(double));
  // P takes the first 16 MiB (K R^2 <= 4,194,304); the rest (< 1.2 MiB for R <= 64) follows
  if ((int64_t)K * RR > (int64_t)DPAR2_NOALLOC_MAX_KRR || bP + bD + bA + bF > (size_t)DPAR2_NOALLOC_SCRATCH_BYTES) {
    ctx->err = "K R^2 = " + std::to_string((int64_t)K * RR) + " is above " +
               std::to_string((int64_t)DPAR2_NOALLOC_MAX_KRR) + ", the limit of the fixed " +
               std::to_string((size_t)DPAR2_NOALLOC_SCRATCH_BYTES) + "-byte scratch (use dpar2_reconstruct_error)";
    return DPAR2_ERR_INVALID_ARG;
  }
  double res[2] = {0, 0};
  dpar2_status st = guarded(ctx, stream, [&](cudaStream_t s) {
    unsigned char* base = static_cast<unsigned char*>(noalloc_base());
    float* P = reinterpret_cast<float*>(base);
    double* Psi = reinterpret_cast<double*>(base + bP);
    double* VtV = Psi + RR;
    float* apart = reinterpret_cast<float*>(base + bP + bD);
    double* fpart = reinterpret_cast<double*>(base + bP + bD + bA);
    launch_psi_vtv(J, R, static_cast<const float*>(comp->D.p), V, Psi, VtV, apart, s);
    launch_vtm(K, J, R, V, comp->M.p, (int64_t)K * R * comp->Jq, comp->Jq, P, s);
    launch_fitness(K, R, P, Upol, H, W, VtV, static_cast<const double*>(comp->xnorm2.p), fpart, nblk, fpart + nblk,
                   s);
    DP2_COUNTED(k_sum_f64<<<1, 256, 0, s>>>(static_cast<const double*>(comp->xnorm2.p), K, fpart + nblk + 1));
    CK(cudaMemcpyAsync(res, fpart + nblk, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
  });
  if (st == DPAR2_OK) {
    if (sq_err) *sq_err = res[0];
    if (fitness) *fitness = res[1] > 0 ? 1.0 - res[0] / res[1] : 0.0;
  }
  return st;
}

// ------------------------------------------------------------ comp access ----
size_t dpar2_comp_bytes(const dpar2_comp* c) {
  if (!c) return 0;
  return 4 * ((size_t)c->N * c->R + (size_t)c->K * c->R * c->R + (size_t)c->J * c->R + c->R);
}
size_t dpar2_comp_device_bytes(const dpar2_comp* c) { return c ? c->device_bytes() : 0; }

dpar2_status dpar2_comp_view_get(const dpar2_comp* c, dpar2_comp_view* v) {
  if (!c || !v) return DPAR2_ERR_INVALID_ARG;
  v->K = c->K;
  v->J = c->J;
  v->R = c->R;
  v->ell = c->ell;
  v->N = c->N;
  v->offsets = static_cast<const int64_t*>(c->offsets.p);
  v->A = static_cast<const float*>(c->A.p);
  v->Bk = static_cast<const float*>(c->Bk.p);
  v->Jq = c->Jq;
  v->Ms = c->M.p;
  v->D = static_cast<const float*>(c->D.p);
  v->E = static_cast<const float*>(c->E.p);
  v->Ft = static_cast<const float*>(c->Ft.p);
  v->xnorm2 = static_cast<const double*>(c->xnorm2.p);
  v->rank1 = static_cast<int32_t*>(c->rank1.p);
  return DPAR2_OK;
}

dpar2_status dpar2_projection_config(const dpar2_ctx* ctx, int* schedule, int* cols) {
  if (!ctx || !schedule || !cols) return DPAR2_ERR_INVALID_ARG;
  *schedule = ctx->pj_last_schedule;
  *cols = ctx->pj_last_cols;
  return DPAR2_OK;
}

dpar2_status dpar2_comp_m(dpar2_ctx* ctx, const dpar2_comp* comp, float* M, void* stream) {
  if (!ctx) return DPAR2_ERR_INVALID_ARG;
  if (!comp || !M || !comp->M.p) {
    ctx->err = "comp and M must be non-null and the compression must hold M";
    return DPAR2_ERR_INVALID_ARG;
  }
  return guarded(ctx, stream, [&](cudaStream_t s) {
    launch_ms_to_m(comp->M.p, (int64_t)comp->K * comp->R * comp->Jq, comp->K, comp->J, comp->Jq, comp->R, M, s);
  });
}

void dpar2_comp_free(dpar2_comp* c) {
  if (!c) return;
  int prev = -1;
  cudaGetDevice(&prev);
  dpar2_ctx* owner = c->owner;
  if (owner) cudaSetDevice(owner->device);
  cudaDeviceSynchronize();  // work of any stream that still reads the object
  delete c;
  if (owner && --owner->live_comps == 0 && owner->closing) ctx_release(owner);
  if (prev >= 0) cudaSetDevice(prev);
}

// ------------------------------------------------------- learned sketch ----
dpar2_status dpar2_sketch_loss_fwd(dpar2_ctx* ctx, int K, int J, const int64_t* row_offsets, const void* X,
                                   int64_t ldx, dpar2_dtype dtype, const float* omega, int ell, double* loss,
                                   void* stream) {
  if (!ctx) return DPAR2_ERR_INVALID_ARG;
  try {
    require(X && row_offsets && omega && loss, DPAR2_ERR_INVALID_ARG, "X, row_offsets, omega and loss must be non-null");
    require(dtype == DPAR2_F32 || dtype == DPAR2_BF16 || dtype == DPAR2_F16, DPAR2_ERR_INVALID_ARG, "bad dtype");
    require(K >= 1 && J >= 1, DPAR2_ERR_SHAPE, "K and J must be >= 1");
    require(ell >= 1 && ell <= std::min(J, kMaxEll), DPAR2_ERR_SHAPE, "need 1 <= l <= min(J, 64)");
    require(ldx >= J, DPAR2_ERR_SHAPE, "ldx < J");
    require((ldx * (int64_t)dtype_size(dtype)) % 16 == 0, DPAR2_ERR_INVALID_ARG,
            "ldx * sizeof(dtype) must be a multiple of 16 bytes");
    require((reinterpret_cast<uintptr_t>(X) & 15) == 0, DPAR2_ERR_INVALID_ARG, "X must be 16-byte aligned");
    require(row_offsets[0] == 0, DPAR2_ERR_SHAPE, "row_offsets[0] must be 0");
    for (int k = 0; k < K; ++k)
      require(row_offsets[k + 1] > row_offsets[k], DPAR2_ERR_SHAPE, "every slice needs I_k >= 1 rows");
  } catch (const Fail& f) {
    ctx->err = f.msg;
    return f.st;
  }
  ctx->sk_ready = false;
  double* h_loss = nullptr;
  dpar2_status st = guarded(ctx, stream, [&](cudaStream_t s) {
    const int LP = round_up(ell, 8), Jp = round_up(J, 4), Jpad = round_up(J, 32);
    const int64_t N = row_offsets[K];
    int64_t maxI = 0;
    for (int k = 0; k < K; ++k) maxI = std::max<int64_t>(maxI, row_offsets[k + 1] - row_offsets[k]);
    const bool use_tc = dtype != DPAR2_F32 && tc_available();
    const int LPN = tc_lpn(ell);
    ctx->sk_K = K;
    ctx->sk_J = J;
    ctx->sk_ell = ell;
    ctx->sk_LP = LP;
    ctx->sk_N = N;
    ctx->sk_ldx = ldx;
    ctx->sk_maxI = maxI;
    ctx->sk_X = X;
    ctx->sk_dtype = dtype;
    ctx->sk_tc = use_tc;
    int64_t* d_off = wsget<int64_t>(ctx, "sl_off", (size_t)K + 1);
    h2d_i64(ctx, d_off, row_offsets, (K + 1), s);

    // pass 1: Y = X Omega (Omega rounded to X's 16-bit type, as in dpar2_compress)
    float* om_pad = wsget<float>(ctx, "sl_om_pad", (size_t)Jpad * LP);
    launch_pad_omega(omega, J, ell, Jpad, LP, dtype, om_pad, s);
    float* Y = wsget<float>(ctx, "sl_Y", (size_t)N * LP);
    bool done = false;
    if (use_tc) {
      void* omT16 = wsget<uint16_t>(ctx, "sl_omT16", (size_t)LPN * Jpad);
      launch_omega_t16(om_pad, Jpad, LP, LPN, dtype, omT16, s);
      done = launch_sketch_tc(X, dtype, ldx, N, J, omT16, Jpad, LPN, LP, Y, ctx->num_sms, ctx->d_status, s);
      require(done, DPAR2_ERR_CUDA, "tensor map encoding failed");
    } else {
      launch_sketch_generic(X, dtype, ldx, N, J, om_pad, LP, Y, s);
    }
    // CholeskyQR2: Y <- Q1 = Y M1, M2 (Q = Q1 M2)
    float* M2 = wsget<float>(ctx, "sl_M2", (size_t)K * LP * LP);
    cholqr2(ctx, Y, d_off, K, maxI, ell, LP, M2, wsget<int>(ctx, "sl_rank", (size_t)K), s, "sl");
    // pass 2: B1 = Q1^T X and ||X_k||^2
    float* B1 = wsget<float>(ctx, "sl_B1", (size_t)K * LP * Jp);
    double* xn = wsget<double>(ctx, "sl_xn", (size_t)K);
    if (use_tc) {
      std::vector<int64_t>& hp = ctx->sk_poff;
      hp.assign(K + 1, 0);
      int64_t maxPad = 0;
      for (int k = 0; k < K; ++k) {
        const int64_t pk = round_up64(row_offsets[k + 1] - row_offsets[k], 64);
        hp[k + 1] = hp[k] + pk;
        maxPad = std::max(maxPad, pk);
      }
      int64_t* d_poff = wsget<int64_t>(ctx, "sl_poff", (size_t)K + 1);
      h2d_i64(ctx, d_poff, hp.data(), (K + 1), s);
      int PNS = 0, POFF = 0;
      proj_layout(ell, &PNS, &POFF);
      void* Qs = wsget<uint16_t>(ctx, "sl_Qs", (size_t)PNS * hp[K]);
      launch_qsplit(Y, LP, PNS, POFF, d_off, d_poff, K, hp[K], maxPad, dtype, Qs, s);
      const int nJb = (Jp + project_tc_cols(PNS) - 1) / project_tc_cols(PNS);
      double* xp = wsget<double>(ctx, "sl_xpart_tc", (size_t)K * nJb * kProjNormWarps);
      done = launch_project_tc(X, dtype, ldx, N, d_off, d_poff, K, J, Jp, Qs, hp[K], PNS, POFF, LP, B1, xp, nJb, true,
                               ctx->num_sms, ctx->d_status, s);
      require(done, DPAR2_ERR_CUDA, "tensor map encoding failed");
      launch_reduce_rows_f64(xp, K, nJb * kProjNormWarps, xn, s);
    } else {
      const int nJb = project_blocks(Jp, LP);
      double* xp = wsget<double>(ctx, "sl_xpart", (size_t)K * nJb);
      launch_project_generic(X, dtype, ldx, d_off, K, J, Jp, Y, LP, B1, xp, nullptr, s);
      launch_reduce_rows_f64(xp, K, nJb, xn, s);
    }
    // ||Q_k^T X_k||^2 = tr(M2^T GB M2), GB = B1 B1^T
    double* GB = wsget<double>(ctx, "sl_GB", (size_t)K * LP * LP);
    launch_gram_b1(B1, Jp, J, K, ell, LP, GB, s);
    double* dl = wsget<double>(ctx, "sl_loss", 2);
    const float* M1 = wsget<float>(ctx, "sl_M1", (size_t)K * LP * LP);
    float* P = wsget<float>(ctx, "sl_P", (size_t)K * LP * LP);
    float* S = wsget<float>(ctx, "sl_S", (size_t)K * LP * LP);
    launch_sl_loss(M1, M2, GB, xn, K, ell, LP, wsget<double>(ctx, "sl_ratio", (size_t)K), P, S, dl, s);
    h_loss = reinterpret_cast<double*>(ctx->h_status) + 1;
    CK(cudaMemcpyAsync(h_loss, dl, sizeof(double), cudaMemcpyDeviceToHost, s));
    // row ranges of the gradient's last pass, 64-row aligned: about one per SM,
    // a multiple of the tensor-core projection's teams (num_sms / column blocks)
    const int nJb_g = (Jp + project_tc_cols(3 * LPN) - 1) / project_tc_cols(3 * LPN);
    const int nteam = std::max(1, ctx->num_sms / nJb_g);
    const int64_t want = std::max<int64_t>(1, std::min<int64_t>(nteam * std::max(1, ctx->num_sms / nteam),
                                                                (N + 63) / 64));
    const int64_t per = round_up64((N + want - 1) / want, 64);
    ctx->sk_off2.clear();
    for (int64_t r = 0; r < N; r += per) ctx->sk_off2.push_back(r);
    ctx->sk_off2.push_back(N);
    ctx->sk_toff.assign(K + 1, 0);
    for (int k = 0; k < K; ++k)
      ctx->sk_toff[k + 1] = ctx->sk_toff[k] + (row_offsets[k + 1] - row_offsets[k] + 127) / 128;
  });
  if (st == DPAR2_OK) {
    *loss = *h_loss;
    ctx->sk_ready = true;
  }
  return st;
}

dpar2_status dpar2_sketch_loss_bwd(dpar2_ctx* ctx, double grad_scale, float* grad_omega, void* stream) {
  if (!ctx) return DPAR2_ERR_INVALID_ARG;
  if (!grad_omega) {
    ctx->err = "grad_omega must be non-null";
    return DPAR2_ERR_INVALID_ARG;
  }
  if (!ctx->sk_ready) {
    ctx->err = "dpar2_sketch_loss_bwd needs a successful dpar2_sketch_loss_fwd on this context first";
    return DPAR2_ERR_INVALID_ARG;
  }
  return guarded(ctx, stream, [&](cudaStream_t s) {
    const int K = ctx->sk_K, J = ctx->sk_J, ell = ctx->sk_ell, LP = ctx->sk_LP;
    const int Jp = round_up(J, 4), Jpad = round_up(J, 32), LPN = tc_lpn(ell);
    const int64_t N = ctx->sk_N, maxI = ctx->sk_maxI;
    const dpar2_dtype dtype = ctx->sk_dtype;
    const void* X = ctx->sk_X;
    const int64_t* d_off = wsget<int64_t>(ctx, "sl_off", (size_t)K + 1);
    const float* Q1 = wsget<float>(ctx, "sl_Y", (size_t)N * LP);
    const float* B1 = wsget<float>(ctx, "sl_B1", (size_t)K * LP * Jp);
    const double* xn = wsget<double>(ctx, "sl_xn", (size_t)K);
    const float* P = wsget<float>(ctx, "sl_P", (size_t)K * LP * LP);
    const float* S = wsget<float>(ctx, "sl_S", (size_t)K * LP * LP);
    float* sk = wsget<float>(ctx, "sl_opscale", (size_t)K * LP);

    // pass 3: V_k = X_k B1_k^T (W applies P_k: V_k P_k = X_k Mk)
    float* U = wsget<float>(ctx, "sl_U", (size_t)N * LP);
    if (ctx->sk_tc) {
      void* Ms = wsget<uint16_t>(ctx, "sl_Ms", (size_t)K * 3 * LPN * Jpad);
      launch_sl_rowsplit(B1, K, Jp, J, Jpad, ell, LP, LPN, dtype, Ms, nullptr, sk, s);
      int64_t* d_toff = wsget<int64_t>(ctx, "sl_toff", (size_t)K + 1);
      h2d_i64(ctx, d_toff, ctx->sk_toff.data(), (K + 1), s);
      const bool ok = launch_sketch_seg_tc(X, dtype, ctx->sk_ldx, N, J, d_off, d_toff, ctx->sk_toff[K], K, Ms, Jpad,
                                           LPN, LP, U, ctx->num_sms, ctx->d_status, s);
      require(ok, DPAR2_ERR_CUDA, "tensor map encoding failed");
    } else {
      float* omk = wsget<float>(ctx, "sl_omk", (size_t)K * Jpad * LP);
      launch_sl_rowsplit(B1, K, Jp, J, Jpad, ell, LP, LPN, dtype, nullptr, omk, sk, s);
      launch_sketch_generic_per_slice(X, dtype, ctx->sk_ldx, d_off, K, (int)maxI, J, omk, Jpad, LP, U, s);
    }

    // W_k = c_k (U_k - Q1_k S_k); pass 4: grad^T = sum over row ranges of W^T X
    const int np = (int)ctx->sk_off2.size() - 1;
    int64_t* d_off2 = wsget<int64_t>(ctx, "sl_off2", (size_t)np + 1);
    h2d_i64(ctx, d_off2, ctx->sk_off2.data(), (np + 1), s);
    float* GP = wsget<float>(ctx, "sl_GP", (size_t)np * LP * Jp);
    float* Wf = wsget<float>(ctx, "sl_W", (size_t)N * LP);
    unsigned* wmax = wsget<unsigned>(ctx, "sl_wmax", (size_t)LP);
    float* bmax = wsget<float>(ctx, "sl_bmax", (size_t)sl_wrows_blocks(K, maxI) * LP);
    launch_sl_wrows(U, Q1, d_off, K, maxI, LP, P, S, xn, grad_scale, sk, Wf, bmax, wmax, s);
    if (ctx->sk_tc) {
      const int64_t Npad = round_up64(N, 64);
      ctx->sk_poff2 = ctx->sk_off2;
      ctx->sk_poff2[np] = Npad;
      int64_t* d_poff2 = wsget<int64_t>(ctx, "sl_poff2", (size_t)np + 1);
      h2d_i64(ctx, d_poff2, ctx->sk_poff2.data(), (np + 1), s);
      uint16_t* Ws = wsget<uint16_t>(ctx, "sl_Ws", (size_t)3 * LPN * Npad);
      if (N % 64) CK(cudaMemsetAsync(Ws + (N / 64) * 3 * LPN * 64, 0, (size_t)3 * LPN * 64 * 2, s));
      launch_sl_wsplit(Wf, N, LP, LPN, wmax, dtype, Ws, s);
      // W's split has the standard layout: parts LPN rows apart, N = 3 LPN
      const int nJb = (Jp + project_tc_cols(3 * LPN) - 1) / project_tc_cols(3 * LPN);
      double* xp = wsget<double>(ctx, "sl_xpart2", (size_t)np * nJb * kProjNormWarps);
      const bool ok = launch_project_tc(X, dtype, ctx->sk_ldx, N, d_off2, d_poff2, np, J, Jp, Ws, Npad, 3 * LPN, LPN, LP, GP,
                                        xp, nJb, false, ctx->num_sms, ctx->d_status, s);
      require(ok, DPAR2_ERR_CUDA, "tensor map encoding failed");
    } else {
      launch_project_generic(X, dtype, ctx->sk_ldx, d_off2, np, J, Jp, Wf, LP, GP, nullptr, nullptr, s);
    }
    launch_sl_gradsum(GP, np, LP, Jp, J, ell, ctx->sk_tc ? wmax : nullptr, grad_omega, s);
  });
}

dpar2_status dpar2_orthonormalize(dpar2_ctx* ctx, int64_t rows, int cols, float* A, void* stream) {
  if (!ctx) return DPAR2_ERR_INVALID_ARG;
  if (!A || cols < 1 || cols > kMaxEll || rows < cols) {
    ctx->err = "need A non-null and 1 <= cols <= min(rows, 64)";
    return A ? DPAR2_ERR_SHAPE : DPAR2_ERR_INVALID_ARG;
  }
  return guarded(ctx, stream, [&](cudaStream_t s) {
    const int LP = round_up(cols, 8);
    float* Y = wsget<float>(ctx, "on_Y", (size_t)rows * LP);
    launch_pad_omega(A, (int)rows, cols, (int)rows, LP, DPAR2_F32, Y, s);
    int64_t* d_off = wsget<int64_t>(ctx, "on_off", 2);
    const int64_t hoff[2] = {0, rows};
    h2d_i64(ctx, d_off, hoff, sizeof(hoff) / sizeof(int64_t), s);
    float* M2 = wsget<float>(ctx, "on_M2", (size_t)LP * LP);
    cholqr2(ctx, Y, d_off, 1, rows, cols, LP, M2, wsget<int>(ctx, "on_rank", 1), s, "on");
    DP2_COUNTED(k_apply_m2<<<dim3((unsigned)((rows + 127) / 128), 1), 128, 0, s>>>(Y, d_off, LP, M2));
    CK(cudaMemcpy2DAsync(A, cols * sizeof(float), Y, LP * sizeof(float), cols * sizeof(float), rows,
                         cudaMemcpyDeviceToDevice, s));
  });
}

// ------------------------------------------------------- post-fit analyses --
dpar2_status dpar2_similarity(dpar2_ctx* ctx, int K, int64_t L, const float* U, int64_t ldu, double gamma, float* S,
                              int64_t lds, void* stream) {
  if (!ctx) return DPAR2_ERR_INVALID_ARG;
  if (!U || !S) {
    ctx->err = "U and S must be non-null";
    return DPAR2_ERR_INVALID_ARG;
  }
  if (K < 1 || L < 1 || ldu < L || lds < K || L > (int64_t)1 << 30 || !(gamma >= 0.0)) {
    ctx->err = "need K >= 1, L >= 1, ldu >= L, lds >= K and gamma >= 0";
    return DPAR2_ERR_SHAPE;
  }
  if (!tc_available()) {
    ctx->err = "tensor-map encoding unavailable (driver entry point cuTensorMapEncodeTiled)";
    return DPAR2_ERR_UNSUPPORTED;
  }
  return guarded(ctx, stream, [&](cudaStream_t s) {
    const int ldp = round_up((int)L, 8);
    void* parts = wsget<uint16_t>(ctx, "sim_parts", (size_t)3 * K * ldp);
    double* nrm = wsget<double>(ctx, "sim_nrm", (size_t)K);
    if (!launch_similarity(K, (int)L, U, ldu, gamma, S, lds, parts, ldp, nrm, ctx->num_sms, ctx->d_status, s))
      throw Fail{DPAR2_ERR_UNSUPPORTED, "tensor map creation failed"};
  });
}

dpar2_status dpar2_topk(dpar2_ctx* ctx, int nrows, int n, const float* scores, int64_t ld, const int* exclude, int k,
                        int* idx, float* val, void* stream) {
  if (!ctx) return DPAR2_ERR_INVALID_ARG;
  if (!scores || !idx || !val) {
    ctx->err = "scores, idx and val must be non-null";
    return DPAR2_ERR_INVALID_ARG;
  }
  if (nrows < 1 || n < 1 || ld < n || k < 1 || k > 16) {
    ctx->err = "need nrows >= 1, n >= 1, ld >= n and 1 <= k <= 16";
    return DPAR2_ERR_SHAPE;
  }
  return guarded(ctx, stream, [&](cudaStream_t s) {
    int* dex = nullptr;
    if (exclude) {
      std::vector<int32_t> hx(exclude, exclude + nrows);
      dex = wsget<int>(ctx, "topk_ex", (size_t)nrows);
      h2d_bytes(ctx, dex, hx.data(), (size_t)nrows * sizeof(int32_t), s);
    }
    launch_topk(nrows, n, scores, ld, dex, k, idx, val, s);
  });
}

dpar2_status dpar2_rwr(dpar2_ctx* ctx, int K, const float* S, int64_t lds, int nq, const int* targets, double c,
                       int iters, float* r, void* stream) {
  if (!ctx) return DPAR2_ERR_INVALID_ARG;
  if (!S || !targets || !r) {
    ctx->err = "S, targets and r must be non-null";
    return DPAR2_ERR_INVALID_ARG;
  }
  if (K < 2 || lds < K || nq < 1 || nq > rwr_max_queries() || iters < 0 || !(c >= 0.0 && c <= 1.0)) {
    ctx->err = "need K >= 2, lds >= K, 1 <= nq <= 16, iters >= 0 and 0 <= c <= 1";
    return DPAR2_ERR_SHAPE;
  }
  for (int q = 0; q < nq; ++q)
    if (targets[q] < 0 || targets[q] >= K) {
      ctx->err = "targets must lie in [0, K)";
      return DPAR2_ERR_SHAPE;
    }
  return guarded(ctx, stream, [&](cudaStream_t s) {
    std::vector<int32_t> ht(targets, targets + nq);
    int* dt = wsget<int>(ctx, "rwr_tgt", (size_t)nq);
    h2d_bytes(ctx, dt, ht.data(), (size_t)nq * sizeof(int32_t), s);
    double* deg = wsget<double>(ctx, "rwr_deg", (size_t)K);
    float* y0 = wsget<float>(ctx, "rwr_y0", (size_t)K * rwr_max_queries());
    float* y1 = wsget<float>(ctx, "rwr_y1", (size_t)K * rwr_max_queries());
    launch_rwr(K, S, lds, nq, dt, c, iters, deg, r, y0, y1, s);
  });
}

dpar2_status dpar2_feature_pcc(dpar2_ctx* ctx, int J, int R, const float* V, float* C, void* stream) {
  if (!ctx) return DPAR2_ERR_INVALID_ARG;
  if (!V || !C) {
    ctx->err = "V and C must be non-null";
    return DPAR2_ERR_INVALID_ARG;
  }
  if (J < 1 || R < 2) {
    ctx->err = "need J >= 1 and R >= 2";
    return DPAR2_ERR_SHAPE;
  }
  return guarded(ctx, stream, [&](cudaStream_t s) {
    float* Vn = wsget<float>(ctx, "pcc_vn", (size_t)J * R);
    launch_feature_pcc(J, R, V, Vn, C, s);
  });
}

}  // extern "C"
