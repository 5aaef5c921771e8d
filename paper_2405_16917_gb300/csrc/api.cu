#include <map>
#include <mutex>
#include <atomic>
// C ABI of the LRAMM library: plan, workspace layout and the pipeline
//   RSVD(A), RSVD(B)  (Sec. 2.2 range finder + Algorithm 1)
//   E1, E2, E3 chain  (Algorithm 3, QM of Algorithm 2)
// Every kernel is enqueued on the caller's stream; nothing here allocates
// device memory or synchronises (except lramm_status_read).
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <new>
#include <vector>

#include <algorithm>

#include "common.cuh"

using namespace lramm;

namespace lramm {
static thread_local char g_cuda_err[256];
static std::atomic<unsigned long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

void note_cuda_error(cudaError_t e, const char* where) {
  snprintf(g_cuda_err, sizeof(g_cuda_err), "%s: %s (%s)", where, cudaGetErrorName(e), cudaGetErrorString(e));
}

int num_sms() {
  constexpr int kMaxDev = 64;
  static std::atomic<int> cache[kMaxDev];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return 152;
  int v = cache[dev].load(std::memory_order_relaxed);
  if (v > 0) return v;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v < 1) v = 152;
  cache[dev].store(v, std::memory_order_relaxed);
  return v;
}

cudaError_t smem_cap_fn(const void* fn, size_t need) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, size_t> caps;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  auto it = caps.find({fn, dev});
  if (it == caps.end()) {
    cudaFuncAttributes fa{};
    int optin = 0;
    if ((e = cudaFuncGetAttributes(&fa, fn)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess) return e;
    const size_t cap = static_cast<size_t>(optin) > fa.sharedSizeBytes ? optin - fa.sharedSizeBytes : 0;
    if ((e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(cap))) !=
        cudaSuccess)
      return e;
    it = caps.emplace(std::make_pair(fn, dev), cap).first;
  }
  return need <= it->second ? cudaSuccess : cudaErrorInvalidValue;
}
}  // namespace lramm

namespace {

constexpr size_t kAlign = 256;
constexpr int kStatusWords = 24;   // status-area words cleared at the start of a call
constexpr int kMaxL = 576;   // the SVD form stops earlier, at jacobi_max_l()

// Largest l of the small SVD (the SVD form); the range-finder form needs none.
int svd_max_l() {
  static const int v = jacobi_max_l();
  return v;
}
constexpr float kCholShift = 4.0f * 0x1p-24f;  // relative diagonal shift of every CholeskyQR pass
// Jacobi stopping multipliers (of tol = 4 sqrt(l) u): a sweep whose largest
// relative inner product rho is below the multiplier times tol is the last.
// 20: the converged SVD the rank-r factors of lramm_rsvd / lramm_qsvd and the
// FP32 chains use (the next sweep would rotate nothing).  1000 (rho below
// 3.9e-3 at l = 272): the factors of quantised chains inside lramm_matmul --
// the relative inner products left after such a sweep are about 5 rho^2
// (the next sweep's rho), which moves the rank-r product by about ten times
// that in the M-only form these chains use (first order in the leftover;
// with V_s accumulated it would be second order), <= 1e-3 relative, below
// the code noise of an 8-bit chain.
constexpr float kJacobiQuad = 20.0f;
constexpr float kJacobiQuadQuantised = 1000.0f;
constexpr int64_t kGramTcRows = 2048;          // sketches from this many rows take the tensor-core Gram

struct SideLayout {
  int64_t rows, cols;
  size_t omega, R0, R1, C0, C1, G, L1, L2, L3, Xd, Lh, Ll, R, Vj, sig, S1, S2, S1T, S2T, CS;
  size_t part, gpart, gtpart, bsplit;   // this operand's split-K partials and BF16 parts (own stream)
  // E4M3 range finder: codes of X per row (rows x cols_p) and per column
  // (cols x rows_p), of the l-column operand (l x max(rows_p, cols_p)), their
  // scales, column a_max scratch and the products' split-K partials
  size_t xc, xs, xtc, xts, bc, bs, cam, qp, qp_floats;
};

}  // namespace

struct TimerRec {
  int kind;
  cudaEvent_t a, b;
};

struct lramm_plan_s {
  lramm_desc d;
  bool timing = false;
  std::vector<TimerRec> recs;
  size_t used = 0;
  int l;
  int64_t kp, rp;
  SideLayout side[2];
  size_t Ut, Vt, Wt, Zt, E1, E2t;
  size_t cV, cW, cE1, cZ, cU, cE2;
  size_t sV, sW, sE1, sZ, sU, sE2;
  size_t amax, amax2;   // per-tensor amax words: the call's stream, and the second operand's stream
  size_t qpart;
  size_t bsplit_bytes;           // BF16 parts of the l-column operand (BF16 A or B), per side
  // second stream and fork / join events: the two operands' RSVDs overlap
  cudaStream_t s2 = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaEvent_t ev_stag = nullptr;   // B's first product waits for A's (staggered chains)
  int dev = -1;
  // LRAMM_FLAG_GRAPH: the captured call and the arguments it was captured with
  cudaGraphExec_t gexec = nullptr;
  const void* gkey[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  int gdev = -1;
  size_t glaunches = 0;   // kernels in the captured graph
  // MXFP4 block exponents of the chain operands; the lead / tail E3 buffers
  size_t xV, xW, xZ, xE1, xU, xE2;
  int64_t lq;
  size_t cUh, cUl, cEh, cEl, sUh, sUl, sEh, sEl, tres;
  size_t vU, vE;   // MXFP4 E3 operands as exact BF16 values (m x rp, n x rp); 0 when unused
  size_t xT, xP;
  size_t qpart_floats;
  // range-finder form: codes / scales of T and P^T; the range-finder chain
  // kept for the backward (Q_0..Q_q, Z_1..Z_q, the Cholesky factors of every
  // orthonormalisation) and its temporaries
  int64_t lp;
  size_t cT, cP, sT, sP;
  size_t bq, bz, bl;
  size_t tdT, tdP, tdQ, tdZ, tB, tY, tY2, tM, tMc, tI, tLi;
  size_t total;
};

namespace {

struct Bump {
  size_t off = 0;
  size_t take(size_t bytes) {
    const size_t o = off;
    off += (bytes + kAlign - 1) / kAlign * kAlign;
    return o;
  }
};

bool valid_prec(int p) { return p >= LRAMM_P_F32 && p <= LRAMM_P_MXFP4; }

lramm_status validate(const lramm_desc* d) {
  if (!d) return LRAMM_ERR_INVALID_ARG;
  if (d->m < 1 || d->n < 1 || d->k < 1) return LRAMM_ERR_INVALID_ARG;
  if (d->lda < d->k || d->ldb < d->n || d->ldc < d->n) return LRAMM_ERR_INVALID_ARG;
  if ((d->a_type != LRAMM_F32 && d->a_type != LRAMM_BF16) ||
      (d->b_type != LRAMM_F32 && d->b_type != LRAMM_BF16))
    return LRAMM_ERR_INVALID_ARG;
  if (d->r < 1 || d->p < 0 || d->q < 0 || d->q > 16) return LRAMM_ERR_INVALID_ARG;
  const int64_t l = (int64_t)d->r + d->p;
  if (l > d->m || l > d->k || l > d->n) return LRAMM_ERR_INVALID_ARG;
  for (int i = 0; i < 3; ++i)
    if (!valid_prec(d->prec[i])) return LRAMM_ERR_INVALID_ARG;
  if (d->scale != LRAMM_S_ROWCOL && d->scale != LRAMM_S_TENSOR) return LRAMM_ERR_INVALID_ARG;
  if (d->sketch < LRAMM_SKETCH_F32 || d->sketch > LRAMM_SKETCH_E4M3) return LRAMM_ERR_INVALID_ARG;
  if (d->sketch == LRAMM_SKETCH_E4M3 && (d->a_type != LRAMM_F32 || d->b_type != LRAMM_F32))
    return LRAMM_ERR_UNSUPPORTED;
  if (d->max_sweeps < 0 ||
      (d->flags & ~(LRAMM_FLAG_TIMING | LRAMM_FLAG_GRAPH | LRAMM_FLAG_SHORT_WAITS | LRAMM_FLAG_TEST_DROP_MOVE)) != 0)
    return LRAMM_ERR_INVALID_ARG;
  if (d->lead < 0 || d->lead > d->r || d->lead_split < 0 || d->lead_split > 2) return LRAMM_ERR_INVALID_ARG;
  if (d->lead > 0 && d->lead_prec != LRAMM_P_INT8 && d->lead_prec != LRAMM_P_INT4 && d->lead_prec != LRAMM_P_E4M3)
    return LRAMM_ERR_INVALID_ARG;
  if (l > kMaxL) return LRAMM_ERR_UNSUPPORTED;
  // orthonormalisation: blocked Cholesky (l <= 288), two-level beyond
  // (l % 4 == 0), the column-panel Cholesky while its triangle fits
  if (!chol3_supported((int)l) && !chol_split_supported((int)l) && l * (l + 1) / 2 * 4 > 231424)
    return LRAMM_ERR_UNSUPPORTED;
  return LRAMM_OK;
}

void layout(lramm_plan_s* P) {
  const lramm_desc& d = P->d;
  const int64_t l = P->l, r = d.r;
  Bump b;
  b.take(kAlign);  // status word
  for (int s = 0; s < 2; ++s) {
    SideLayout& S = P->side[s];
    S.rows = s == 0 ? d.m : d.k;
    S.cols = s == 0 ? d.k : d.n;
    S.omega = b.take(sizeof(float) * S.cols * l);
    S.R0 = b.take(sizeof(float) * S.rows * l);
    S.R1 = b.take(sizeof(float) * S.rows * l);
    S.C0 = b.take(sizeof(float) * S.cols * l);
    S.C1 = b.take(sizeof(float) * S.cols * l);
    S.G = b.take(sizeof(float) * l * l);
    S.L1 = b.take(sizeof(float) * l * l);
    S.L2 = b.take(sizeof(float) * l * l);
    S.L3 = b.take(sizeof(float) * l * l);
    S.Xd = b.take(sizeof(float) * ceil_div(l, 32) * 32 * 32);
    S.Lh = b.take(sizeof(float) * l * l);   // L^-1 in TF32 parts (tensor-core bases)
    S.Ll = b.take(sizeof(float) * l * l);
    S.CS = chol_split_supported((int)l) ? b.take(sizeof(float) * chol_split_scratch_floats((int)l)) : 0;
    S.R = b.take(sizeof(float) * l * l);
    S.Vj = b.take(sizeof(float) * l * l);
    S.sig = b.take(sizeof(float) * l);
    S.S1 = b.take(sizeof(float) * l * r);
    S.S2 = b.take(sizeof(float) * l * r);
    S.S1T = b.take(sizeof(float) * l * r);
    S.S2T = b.take(sizeof(float) * l * r);
  }
  P->kp = round_up(d.k, 32);   // code rows padded to whole 32-blocks (MXFP4) and 16-K MMA steps
  P->rp = round_up(r, 32);
  P->Ut = b.take(sizeof(float) * d.m * r);
  P->Vt = b.take(sizeof(float) * r * d.k);
  P->Wt = b.take(sizeof(float) * r * d.k);
  P->Zt = b.take(sizeof(float) * d.n * r);
  P->E1 = b.take(sizeof(float) * r * r);
  P->E2t = b.take(sizeof(float) * d.n * r);
  const size_t cb = 2;  // widest code container (bfloat16)
  P->cV = b.take(cb * r * P->kp);
  P->cW = b.take(cb * r * P->kp);
  P->cE1 = b.take(cb * r * P->rp);
  P->cZ = b.take(cb * d.n * P->rp);
  P->cU = b.take(cb * d.m * P->rp);
  P->cE2 = b.take(cb * d.n * P->rp);
  P->sV = b.take(sizeof(float) * r);
  P->sW = b.take(sizeof(float) * r);
  P->sE1 = b.take(sizeof(float) * r);
  P->sZ = b.take(sizeof(float) * d.n);
  P->sU = b.take(sizeof(float) * d.m);
  P->sE2 = b.take(sizeof(float) * d.n);
  P->amax = b.take(kAlign);
  P->amax2 = b.take(kAlign);
  P->xV = b.take(r * (P->kp / 32));
  P->xW = b.take(r * (P->kp / 32));
  P->xE1 = b.take(r * (P->rp / 32));
  P->xZ = b.take(d.n * (P->rp / 32));
  P->xU = b.take(d.m * (P->rp / 32));
  P->xE2 = b.take(d.n * (P->rp / 32));
  P->lq = round_up(d.lead > 0 ? d.lead : 1, 32);
  if (d.lead > 0) {
    P->cUh = b.take(cb * d.m * P->lq);
    P->cUl = b.take(cb * d.m * P->lq);
    P->cEh = b.take(cb * d.n * P->lq);
    P->cEl = b.take(cb * d.n * P->lq);
    P->sUh = b.take(sizeof(float) * d.m);
    P->sUl = b.take(sizeof(float) * d.m);
    P->sEh = b.take(sizeof(float) * d.n);
    P->sEl = b.take(sizeof(float) * d.n);
    P->tres = b.take(sizeof(float) * std::max(d.m, d.n) * d.lead);
  }
  P->vU = d.prec[2] == LRAMM_P_MXFP4 ? b.take(2 * d.m * P->rp) : 0;
  P->vE = d.prec[2] == LRAMM_P_MXFP4 ? b.take(2 * d.n * P->rp) : 0;
  P->bsplit_bytes = (d.a_type == LRAMM_BF16 || d.b_type == LRAMM_BF16)
                        ? sketch_bf_split_bytes(std::max(d.m, std::max(d.k, d.n)), (int)l)
                        : 0;
  for (int sd = 0; sd < 2; ++sd) {   // per operand: the two RSVDs run on two streams
    SideLayout& S = P->side[sd];
    S.part = b.take(sizeof(float) * sketch_tc_part_floats((int)l));
    S.gpart = b.take(sizeof(float) * gram_part_floats((int)l));
    S.gtpart = d.sketch != LRAMM_SKETCH_F32 && gram_tc_supported((int)l)
                   ? b.take(sizeof(float) * gram_tc_part_floats((int)l))
                   : 0;
    S.bsplit = P->bsplit_bytes ? b.take(P->bsplit_bytes) : 0;
    if (d.sketch == LRAMM_SKETCH_E4M3) {
      const int64_t rp = round_up(S.rows, 32), cp = round_up(S.cols, 32);
      S.xc = b.take(S.rows * cp);
      S.xs = b.take(sizeof(float) * S.rows);
      S.xtc = b.take(S.cols * rp);
      S.xts = b.take(sizeof(float) * S.cols);
      S.bc = b.take(l * std::max(rp, cp));
      S.bs = b.take(sizeof(float) * l);
      S.cam = b.take(sizeof(unsigned int) * std::max<int64_t>(S.cols, l));
      S.qp_floats = std::max(qgemm_tc_part_floats(LRAMM_P_E4M3, S.rows, l, cp),
                             qgemm_tc_part_floats(LRAMM_P_E4M3, S.cols, l, rp));
      S.qp = b.take(sizeof(float) * std::max<size_t>(S.qp_floats, 4));
    }
  }
  {  // split-K partials of the tensor-core code products (E1 with long K)
    auto qp = [](int prec, int64_t M, int64_t N, int64_t K) -> size_t {
      return (prec == LRAMM_P_F32 || prec == LRAMM_P_MXFP4) ? 0 : qgemm_tc_part_floats(prec, M, N, K);
    };
    size_t q = qp(d.prec[0], r, r, P->kp);
    q = std::max(q, qp(d.prec[1], d.n, r, P->rp));
    q = std::max(q, qp(d.prec[2], d.m, d.n, P->rp));
    q = std::max(q, qp(d.prec[2], d.m, d.n, round_up(l, 32)));
    if (d.lead > 0) q = std::max(q, qp(d.lead_prec, d.m, d.n, round_up(d.lead, 32)));
    // TF32 products of the range-finder form (K = l)
    q = std::max(q, tgemm_tc_part_floats(d.m, d.n, l));
    q = std::max(q, tgemm_tc_part_floats(d.m, d.k, l));
    q = std::max(q, tgemm_tc_part_floats(d.k, d.n, l));
    P->qpart_floats = q;
    P->qpart = b.take(sizeof(float) * (q > 0 ? q : 4));
  }
  {  // range-finder form
    const int64_t kk = d.k, nn = d.n, mm = d.m, qq = d.q, mx = std::max(kk, nn);
    P->lp = round_up(l, 32);
    P->cT = b.take(cb * mm * P->lp);
    P->cP = b.take(cb * nn * P->lp);
    P->xT = b.take(mm * (P->lp / 32));
    P->xP = b.take(nn * (P->lp / 32));
    P->sT = b.take(sizeof(float) * mm);
    P->sP = b.take(sizeof(float) * nn);
    P->bq = b.take(sizeof(float) * (qq + 1) * kk * l);
    P->bz = b.take(sizeof(float) * std::max<int64_t>(qq, 1) * nn * l);
    P->bl = b.take(sizeof(float) * (2 * qq + 1) * 2 * l * l);
    P->tdT = b.take(sizeof(float) * mm * l);
    P->tdP = b.take(sizeof(float) * nn * l);
    P->tdQ = b.take(sizeof(float) * kk * l);
    P->tdZ = b.take(sizeof(float) * nn * l);
    P->tB = b.take(sizeof(float) * mx * l);
    P->tY = b.take(sizeof(float) * mx * l);
    P->tY2 = b.take(sizeof(float) * mx * l);
    P->tM = b.take(sizeof(float) * l * l);
    P->tMc = b.take(sizeof(float) * l * l);
    P->tI = b.take(sizeof(float) * l * l);
    P->tLi = b.take(sizeof(float) * l * l);
  }
  P->total = b.off;
}

template <typename T>
T* at(void* ws, size_t off) {
  return reinterpret_cast<T*>(static_cast<char*>(ws) + off);
}

// Event pair around one launch when the plan times its calls.
int tbegin(lramm_plan_s* P, int kind, cudaStream_t s) {
  if (!P->timing) return -1;
  if (P->used == P->recs.size()) {
    TimerRec r{kind, nullptr, nullptr};
    if (cudaEventCreate(&r.a) != cudaSuccess || cudaEventCreate(&r.b) != cudaSuccess) return -1;
    P->recs.push_back(r);
  }
  TimerRec& r = P->recs[P->used];
  r.kind = kind;
  if (cudaEventRecord(r.a, s) != cudaSuccess) return -1;
  return (int)P->used++;
}

void tend(lramm_plan_s* P, int h, cudaStream_t s) {
  if (h >= 0) cudaEventRecord(P->recs[h].b, s);
}

#define TIMED(P, kind, s, expr)                  \
  do {                                           \
    const int _h = tbegin((P), (kind), (s));     \
    const lramm_status _st = (expr);             \
    tend((P), _h, (s));                          \
    if (_st != LRAMM_OK) return _st;             \
  } while (0)

lramm_status check_ws(const lramm_plan_s* P, void* ws, size_t ws_bytes) {
  if (!ws || ws_bytes < P->total) return LRAMM_ERR_WORKSPACE;
  if (reinterpret_cast<uintptr_t>(ws) % kAlign) return LRAMM_ERR_WORKSPACE;
  return LRAMM_OK;
}

// X B (a_mn = 0) or X^T B (a_mn = 1) for the range finder: on the tensor
// cores in TF32 when the plan asks for a TF32 sketch and the shapes allow
// (TMA needs l and the row stride of X divisible by 4, 16-byte aligned
// bases), else the FP32 SIMT product.  fp8: a range-finder pass of an E4M3
// plan -- the product of X's e4m3 codes (made by x_codes) with the
// per-column e4m3 codes of B on the tensor cores (kind::f8f6f4), dequantised
// per row of X (or column, for X^T) and per column of B.
lramm_status x_product(lramm_plan_s* P, void* ws, const SideLayout& S, int a_mn, const void* X, int64_t rows,
                       int64_t cols, int64_t ldx, int xbf, const float* B, float* out, cudaStream_t s,
                       bool fp8 = false) {
  const int l = P->l;
  const int sk = P->d.sketch;
  if (fp8 && sk == LRAMM_SKETCH_E4M3) {
    const int64_t rp = round_up(rows, 32), cp = round_up(cols, 32);
    void* bc = at<void>(ws, S.bc);
    float* bs = at<float>(ws, S.bs);
    unsigned int* cam = at<unsigned int>(ws, S.cam);
    if (!a_mn) {   // X B, B cols x l: codes of B's columns as rows (l x cols_p)
      LRAMM_TRY(quantize_cols2d(B, cols, l, l, LRAMM_P_E4M3, bc, cp, bs, cam, s));
      return qgemm_tc(LRAMM_P_E4M3, at<void>(ws, S.xc), bc, rows, l, cp, cp, cp, 1, at<float>(ws, S.xs), bs, 1.f,
                      0.f, nullptr, 0, out, l, at<float>(ws, S.qp), S.qp_floats, at<int>(ws, 0), s);
    }
    // X^T B, B rows x l: codes of B's columns (l x rows_p) against X's column codes
    LRAMM_TRY(quantize_cols2d(B, rows, l, l, LRAMM_P_E4M3, bc, rp, bs, cam, s));
    return qgemm_tc(LRAMM_P_E4M3, at<void>(ws, S.xtc), bc, cols, l, rp, rp, rp, 1, at<float>(ws, S.xts), bs, 1.f, 0.f,
                    nullptr, 0, out, l, at<float>(ws, S.qp), S.qp_floats, at<int>(ws, 0), s);
  }
  if (xbf && sk != LRAMM_SKETCH_F32 && P->bsplit_bytes && sketch_bf_supported(ldx, l, X, B))
    return sketch_bf(a_mn, X, rows, cols, ldx, B, l, sk == LRAMM_SKETCH_TF32 ? 2 : 1, out, at<float>(ws, S.part),
                     sketch_tc_part_floats(l), at<void>(ws, S.bsplit), P->bsplit_bytes, at<int>(ws, 0), s);
  if (sk != LRAMM_SKETCH_F32 && sketch_tc_supported(xbf, ldx, l, X, B))
    return sketch_tc(a_mn, X, rows, cols, ldx, xbf, B, l, out, at<float>(ws, S.part),
                     sketch_tc_part_floats(l), at<int>(ws, 0), s);
  if (a_mn) return sgemm(1, 0, cols, l, rows, 1.f, X, ldx, xbf, B, l, 0.f, out, l, s);
  return sgemm(0, 0, rows, l, cols, 1.f, X, ldx, xbf, B, l, 0.f, out, l, s);
}

// The e4m3 codes of an operand for an E4M3 range finder, once per call:
// per row (rows x cols_p, for X B) and per column (cols x rows_p, for X^T B).
lramm_status x_codes(lramm_plan_s* P, void* ws, const SideLayout& S, const void* X, int64_t ldx, cudaStream_t s) {
  const float* Xf = static_cast<const float*>(X);
  const int64_t rp = round_up(S.rows, 32), cp = round_up(S.cols, 32);
  LRAMM_TRY(quantize_rows(Xf, S.rows, S.cols, ldx, LRAMM_P_E4M3, 1, at<void>(ws, S.xc), cp, at<float>(ws, S.xs),
                          nullptr, s));
  return quantize_cols2d(Xf, S.rows, S.cols, ldx, LRAMM_P_E4M3, at<void>(ws, S.xtc), rp, at<float>(ws, S.xts),
                         at<unsigned int>(ws, S.cam), s);
}

// One operand's share of a randomized SVD run.
struct SideRun {
  const void* X;
  int64_t ldx;
  int xbf;
  const SideLayout* S;
};

// The shifted-CholeskyQR fallback (retry) keeps two words of the status area
// per side: kBrkWord + 2 side (a Cholesky of the current pass met a
// non-positive pivot) and kBrkWord + 2 side + 1 (some pass of this
// orthonormalisation did; the conditional third pass runs).
constexpr int kBrkWord = 16;
constexpr int kBrkCountWord = 20;   // + side: factorisations of this call that broke down (diagnostics)

// Relative diagonal shift of the fallback's factorisation: above the rounding
// error of an l x l Cholesky (~l u) and of the Gram of `rows` rows
// (~sqrt(rows) u), so that it succeeds for a numerically rank-deficient Y.
float chol_shift_big(int64_t rows, int l) {
  return 0x1p-24f * (16.0f * static_cast<float>(l) + 8.0f * sqrtf(static_cast<float>(rows)));
}

// Orthonormalise, for every side s, the rows_s x l matrix src[s] (stride l)
// by `passes` CholeskyQR passes (Gram, Cholesky, Q = Y L^-T); every pass
// shifts the Gram diagonal by 4u max(diag) so a rank-deficient sketch still
// factors (the shift costs ~4u in orthonormality).  One pass suffices where
// only the span matters (the intermediate bases of the power iterations);
// two give orthonormality to working precision.  dst may equal src.  With
// want_R (two passes): R = L2^T L1^T, so that src = dst R.
// skip_last_solve: the last pass forms its Gram and Cholesky factor (and R)
// but not its orthonormal output, so dst keeps what it held (with passes = 2
// and dst = src: the input X, with X = P1 R1 and P1 in tmp).
//
// retry (one side; the blocked and two-level Cholesky paths): the shifted
// CholeskyQR fallback for sketches too ill-conditioned for the 4u shift.  A
// Cholesky that meets a non-positive pivot is redone with the shift
// chol_shift_big (inside the blocked kernel; by a launch predicated on the
// breakdown word for the two-level one), which always factors; the pass's Q
// then spans Y with a condition number near 1 / sqrt(that shift).  With FP32
// products and passes = 2 a third pass, predicated on the same event,
// restores orthonormality to working precision (shifted CholeskyQR3), R
// becoming L3^T L2^T L1^T.  With tensor-core products (TF32 / BF16 parts /
// e4m3) the second pass already leaves an orthogonality error near
// u / shift < 2^-12, below those products' own rounding, and no third pass
// is enqueued.  Without a breakdown the predicated launches do nothing and
// the results are those of the plain passes.
lramm_status orth_sides(lramm_plan_s* P, void* ws, const SideRun* sd, int ns, float* const* src,
                        float* const* tmp, float* const* dst, const int64_t* rows, int passes, bool want_R,
                        int* st, cudaStream_t s, bool skip_last_solve = false, bool retry = false) {
  const int l = P->l;
  const bool c3 = chol3_supported(l) && l % 4 == 0;
  const bool csplit = !c3 && chol_split_supported(l);
  retry = retry && ns == 1 && (c3 || csplit);
  const bool third = retry && passes == 2 && P->d.sketch == LRAMM_SKETCH_F32;
  // tensor-core range finders: the bases Q = Y L^-T by the split-TF32
  // product with L^-1 (accuracy of the split-TF32 Gram); FP32 range finders
  // keep the FP32 panel solve
  const bool tcb = P->d.sketch != LRAMM_SKETCH_F32 && basis_tc_supported(l);
  int* brk = nullptr;
  int* any = nullptr;
  if (retry) {
    brk = at<int>(ws, 0) + kBrkWord + 2 * (sd[0].S == &P->side[1] ? 1 : 0);
    any = brk + 1;
    // (a blocked single pass needs neither word: its restart is internal)
    if (csplit || third) LRAMM_CUDA_TRY(cudaMemsetAsync(brk, 0, 2 * sizeof(int), s));
  }
  const int total = passes + (third ? 1 : 0);
  const float* in[2] = {src[0], ns > 1 ? src[1] : nullptr};
  for (int pass = 0; pass < total; ++pass) {
    const bool extra = pass == passes;          // the fallback's third pass: runs after a breakdown only
    const int* cond = extra ? any : nullptr;
    float* out[2];
    SmallBatch cb{}, tb{};
    CholBatch cb3{};
    TrsmBatch tb3{};
    GramBatch gb{};
    cb.n = tb.n = gb.n = cb3.n = tb3.n = ns;
    for (int i = 0; i < ns; ++i) {
      float* G = at<float>(ws, sd[i].S->G);
      float* Lf = at<float>(ws, pass == 0 ? sd[i].S->L1 : (pass == 1 ? sd[i].S->L2 : sd[i].S->L3));
      float* Xd = at<float>(ws, sd[i].S->Xd);
      out[i] = pass >= passes - 1 ? dst[i] : tmp[i];
      gb.p[i] = GramProb{in[i], rows[i], G};
      cb.p[i] = SmallProb{G, Lf, nullptr, 0};
      tb.p[i] = SmallProb{in[i], out[i], Lf, rows[i]};
      cb3.p[i] = CholProb{G, Lf, Xd};
      tb3.p[i] = TrsmProb{in[i], out[i], Lf, Xd, rows[i]};
    }
    // Grams of tall sketches (>= kGramTcRows rows) in split TF32 on the
    // tensor cores when the products already run on them; the rest on the
    // SIMT kernel
    bool tc[2] = {false, false};
    GramBatch gs{};
    for (int i = 0; i < ns; ++i) {
      tc[i] = sd[i].S->gtpart && rows[i] >= kGramTcRows;
      if (!tc[i]) gs.p[gs.n++] = gb.p[i];
    }
    for (int i = 0; i < ns; ++i)
      if (tc[i]) {
        const float* Yi[1] = {in[i]};
        float* Gi[1] = {at<float>(ws, sd[i].S->G)};
        lramm_status gst = LRAMM_OK;
        TIMED(P, LRAMM_K_GRAM, s,
              (gst = gram_tc(1, Yi, &rows[i], Gi, l, at<float>(ws, sd[i].S->gtpart), gram_tc_part_floats(l), st,
                             s, cond)) == LRAMM_ERR_UNSUPPORTED
                  ? [&] {
                      GramBatch g1{};
                      g1.n = 1;
                      g1.p[0] = gb.p[i];
                      return launch_gram(g1, l, at<float>(ws, sd[i].S->gpart), s, cond);
                    }()
                  : gst);
      }
    if (gs.n) TIMED(P, LRAMM_K_GRAM, s, launch_gram(gs, l, at<float>(ws, sd[0].S->gpart), s, cond));
    // the solve: skipped in the last pass with skip_last_solve; with the
    // fallback, the second pass's solve feeds the third and runs with it
    bool solve = true;
    const int* scond = cond;
    if (skip_last_solve) {
      if (extra) solve = false;
      else if (pass == passes - 1) {
        if (third) scond = any;
        else solve = false;
      }
    }
    const bool guard = retry && !extra;   // breakdowns of this pass are retried
    if (c3) {  // blocked Cholesky (restarting itself with the larger shift) + panel solve or inverse
      if (tcb || !solve)   // no panel solve: no inverted diagonal blocks (the inverse forms its own)
        for (int i = 0; i < ns; ++i) cb3.p[i].Xd = nullptr;
      if (guard) {
      cb3.p[0].brk_any = any;
      cb3.p[0].brk_count = at<int>(ws, 0) + kBrkCountWord + (sd[0].S == &P->side[1] ? 1 : 0);
    }
      TIMED(P, LRAMM_K_CHOL, s,
            launch_chol3(cb3, l, kCholShift, st, s, cond, guard ? chol_shift_big(rows[0], l) : 0.f));
      if (solve && tcb) {   // Q = Y L^-T on the tensor cores from the explicit inverse
        LinvBatch lb{};
        lb.n = ns;
        for (int i = 0; i < ns; ++i)
          lb.p[i] = LinvProb{cb3.p[i].L, at<float>(ws, sd[i].S->Lh), at<float>(ws, sd[i].S->Ll)};
        TIMED(P, LRAMM_K_TRSM, s, launch_linv(lb, l, s, scond));
        for (int i = 0; i < ns; ++i)
          TIMED(P, LRAMM_K_TRSM, s, basis_tc(in[i], rows[i], lb.p[i].Lh, lb.p[i].Ll, out[i], l, st, s, scond));
      } else if (solve) {
        TIMED(P, LRAMM_K_TRSM, s, launch_trsm3(tb3, l, s, scond));
      }
    } else if (csplit) {  // two-level Cholesky, same panel solve
      SplitScratch sc{};
      for (int i = 0; i < ns; ++i) sc.w[i] = at<float>(ws, sd[i].S->CS);
      CholBatch cg = cb3;
      if (guard) {
        cg.p[0].brk = brk;
        cg.p[0].brk_any = any;
        cg.p[0].brk_count = at<int>(ws, 0) + kBrkCountWord + (sd[0].S == &P->side[1] ? 1 : 0);
      }
      TIMED(P, LRAMM_K_CHOL, s, launch_chol_split(cg, sc, l, kCholShift, st, s, cond));
      if (guard) {   // redone with the larger shift after a breakdown, then the word cleared
        TIMED(P, LRAMM_K_CHOL, s, launch_chol_split(cb3, sc, l, chol_shift_big(rows[0], l), st, s, brk));
        LRAMM_CUDA_TRY(cudaMemsetAsync(brk, 0, sizeof(int), s));
      }
      if (solve) TIMED(P, LRAMM_K_TRSM, s, launch_trsm3(tb3, l, s, scond));
    } else {
      TIMED(P, LRAMM_K_CHOL, s, launch_chol2(cb, l, kCholShift, st, s));
      if (solve) TIMED(P, LRAMM_K_TRSM, s, launch_trsm_panel(tb, l, s));
    }
    for (int i = 0; i < ns; ++i) in[i] = out[i];
  }
  if (want_R)
    for (int i = 0; i < ns; ++i) {
      const SideLayout& S = *sd[i].S;
      if (passes != 2) return LRAMM_ERR_INVALID_ARG;
      TIMED(P, LRAMM_K_RFACTOR, s,
            sgemm(1, 1, l, l, l, 1.f, at<float>(ws, S.L2), l, 0, at<float>(ws, S.L1), l, 0.f, at<float>(ws, S.R), l,
                  s));
      if (third) {   // after the third pass: R = L3^T (L2^T L1^T), through Vj (free until the small SVD)
        TIMED(P, LRAMM_K_RFACTOR, s,
              sgemm(1, 0, l, l, l, 1.f, at<float>(ws, S.L3), l, 0, at<float>(ws, S.R), l, 0.f, at<float>(ws, S.Vj),
                    l, s, any));
        TIMED(P, LRAMM_K_RFACTOR, s,
              launch_copy_cond(at<float>(ws, S.Vj), at<float>(ws, S.R), static_cast<int64_t>(l) * l, any, s));
      }
    }
  return LRAMM_OK;
}

// One product of the factor assembly: out (M x N, stride ldo) = A B^T with
// A (M x l) and B (N x l) K-major.  For the factors that feed a quantised
// chain inside lramm_matmul (tc: a tensor-core sketch mode, quantised E3;
// with a lead / tail split, E1 and E2 quantised too, so that every term of
// E3 carries their codes' noise) a TF32 tensor-core product with this
// operand's split-K buffer -- its rounding (2^-11 relative) sits far below
// the quantisation step; otherwise (and for the factors lramm_rsvd and
// lramm_qsvd return, orthonormal to working precision) the FP32 SIMT
// product, which takes its operands as given by (ta, Am, lda_s, tb, Bm, ldb_s).
lramm_status assemble(lramm_plan_s* P, void* ws, const SideLayout& S, int64_t M, int64_t N, const float* A,
                      const float* B, float* out, int64_t ldo, int ta, const float* Am, int64_t lda_s, int tb,
                      const float* Bm, int64_t ldb_s, cudaStream_t s, bool tc = false) {
  const int l = P->l;
  const lramm_desc& d = P->d;
  const bool coded = d.lead == 0 || (d.prec[0] != LRAMM_P_F32 && d.prec[1] != LRAMM_P_F32);
  if (tc && d.sketch != LRAMM_SKETCH_F32 && coded && d.prec[2] != LRAMM_P_F32 &&
      tgemm_tc_supported(A, B, l, l, M, N, l) && tgemm_tc_part_floats(M, N, l) <= sketch_tc_part_floats(l)) {
    // info word 3, bit 0: this call assembled a factor on the tensor cores
    LRAMM_CUDA_TRY(cudaMemsetAsync(static_cast<char*>(ws) + 3 * sizeof(int), 1, 1, s));
    return tgemm_tc(M, N, l, 1.f, A, l, B, l, 0.f, out, ldo, at<float>(ws, S.part), sketch_tc_part_floats(l),
                    at<int>(ws, 0), s);
  }
  return sgemm(ta, tb, M, N, l, 1.f, Am, lda_s, 0, Bm, ldb_s, 0.f, out, ldo, s);
}

// Range finder, projection and small SVD of one or two operands in lockstep
// (X rows x cols each).  On exit (workspace, per side): R0 = Q (rows x l),
// C0 = P (cols x l), sig[:r], S1 = U_s[:, :r] (x sigma if s1_sigma[i]),
// S2 = V_s[:, :r] (x sigma if s2_sigma[i]), with X ~ Q U_s diag(sig) V_s^T P^T.
//
// M-only form (m_only_req, one operand, where the M-only Jacobi launches;
// *m_only_done reports it): P is not formed and V_s is not accumulated.
// With B^T = P1 R1 (the first CholeskyQR pass, P1 in C1, R1 = L1^T) and
// R^T = U_s Sigma V_s^T, P V_s = B^T U_s Sigma^-1 = P1 (R1 U_s Sigma^-1).
// On exit C1 = P1 (cols x l), S2 = U_s[:, :r] Sigma^-1 (x sigma if
// s2_sigma) and Vj holds Y^T = S2^T L1 (r x l, FP32): the products P1 Y are
// the right factors P V_s[:, :r] (x sigma).  The small factor Y carries the
// cancellation between R1 and U_s Sigma^-1 in FP32, so the tall product
// with the well-conditioned P1 is as accurate in TF32 as P V_s.  One
// triangular solve fewer, and the Jacobi moves and rotates half the data.
//
// Staggering (two operands on two streams): rec_first is recorded on s after
// this run's first product, and wait_first is waited on before it, so that
// the second operand's chain runs one product behind the first and each
// operand's latency-bound orthonormalisation overlaps the other's
// bandwidth-bound product instead of coinciding with it.
lramm_status rsvd_sides(lramm_plan_s* P, const SideRun* sd, const int* which, int ns, void* ws,
                        const int* s1_sigma, const int* s2_sigma, cudaStream_t s, float stopq = kJacobiQuad,
                        bool m_only_req = false, bool* m_only_done = nullptr, cudaEvent_t rec_first = nullptr,
                        cudaEvent_t wait_first = nullptr) {
  const lramm_desc& d = P->d;
  const int l = P->l;
  const bool fp8 = d.sketch == LRAMM_SKETCH_E4M3;   // range-finder passes on e4m3 codes
  int* st = at<int>(ws, 0);
  float *R0[2], *R1[2], *C0[2], *C1[2];
  int64_t rows[2], cols[2];
  for (int i = 0; i < ns; ++i) {
    const SideLayout& S = *sd[i].S;
    R0[i] = at<float>(ws, S.R0);
    R1[i] = at<float>(ws, S.R1);
    C0[i] = at<float>(ws, S.C0);
    C1[i] = at<float>(ws, S.C1);
    rows[i] = S.rows;
    cols[i] = S.cols;
    float* Om = at<float>(ws, S.omega);
    TIMED(P, LRAMM_K_OMEGA, s, launch_gaussian(d.seed, (uint32_t)which[i], S.cols, l, Om, l, s));
    if (fp8) TIMED(P, LRAMM_K_SKETCH, s, x_codes(P, ws, S, sd[i].X, sd[i].ldx, s));
    if (wait_first) LRAMM_CUDA_TRY(cudaStreamWaitEvent(s, wait_first, 0));
    TIMED(P, LRAMM_K_SKETCH, s,
          x_product(P, ws, *sd[i].S, 0, sd[i].X, S.rows, S.cols, sd[i].ldx, sd[i].xbf, Om, R0[i], s, fp8));
    if (rec_first) LRAMM_CUDA_TRY(cudaEventRecord(rec_first, s));
  }
  LRAMM_TRY(orth_sides(P, ws, sd, ns, R0, R1, R0, rows, d.q > 0 ? 1 : 2, false, st, s, false, true));  // Q
  for (int it = 0; it < d.q; ++it) {
    for (int i = 0; i < ns; ++i)
      TIMED(P, LRAMM_K_SKETCH, s,
            x_product(P, ws, *sd[i].S, 1, sd[i].X, rows[i], cols[i], sd[i].ldx, sd[i].xbf, R0[i], C0[i], s, fp8));
    LRAMM_TRY(orth_sides(P, ws, sd, ns, C0, C1, C0, cols, 1, false, st, s, false, true));  // Z^ (span only)
    for (int i = 0; i < ns; ++i)
      TIMED(P, LRAMM_K_SKETCH, s,
            x_product(P, ws, *sd[i].S, 0, sd[i].X, rows[i], cols[i], sd[i].ldx, sd[i].xbf, C0[i], R0[i], s, fp8));
    LRAMM_TRY(orth_sides(P, ws, sd, ns, R0, R1, R0, rows, it == d.q - 1 ? 2 : 1, false, st, s, false, true));
  }
  for (int i = 0; i < ns; ++i)
    TIMED(P, LRAMM_K_SKETCH, s, x_product(P, ws, *sd[i].S, 1, sd[i].X, rows[i], cols[i], sd[i].ldx, sd[i].xbf, R0[i], C0[i], s));  // B^T
  // R row-major is R^T column-major: one-sided Jacobi on R^T = U_s S V_s^T.
  JacobiBatch jb{};
  FinalBatch fb{};
  jb.n = fb.n = ns;
  jb.info0 = ns == 1 ? which[0] : 0;
  jb.stopq = stopq;
  jb.wait_cycles = (d.flags & LRAMM_FLAG_SHORT_WAITS) ? (1ll << 20) : (1ll << 30);
  jb.drop_rank = (d.flags & LRAMM_FLAG_TEST_DROP_MOVE) ? 1 : -1;
  for (int i = 0; i < ns; ++i) {
    const SideLayout& S = *sd[i].S;
    jb.M[i] = at<float>(ws, S.R);
    jb.V[i] = at<float>(ws, S.Vj);
    fb.p[i] = FinalProb{at<float>(ws, S.R),   at<float>(ws, S.Vj),  at<float>(ws, S.sig),
                        at<float>(ws, S.S1),  at<float>(ws, S.S2),  s1_sigma[i],
                        s2_sigma[i],          at<float>(ws, S.S1T), at<float>(ws, S.S2T)};
  }
  jb.r = d.r;
  for (int i = 0; i < ns; ++i) jb.fin[i] = fb.p[i];
  const int max_sweeps = d.max_sweeps > 0 ? d.max_sweeps : 40;
  bool m_only = false;
  if (m_only_req && ns == 1) LRAMM_TRY(launch_jacobi_uonly(jb, l, max_sweeps, st, s, true, m_only));
  LRAMM_TRY(orth_sides(P, ws, sd, ns, C0, C1, C0, cols, 2, true, st, s, m_only, true));  // B^T = P R
  if (m_only) {
    bool ok = false;
    TIMED(P, LRAMM_K_SVD, s, launch_jacobi_uonly(jb, l, max_sweeps, st, s, false, ok));
    if (!ok) return LRAMM_ERR_UNSUPPORTED;
    const SideLayout& S = *sd[0].S;
    TIMED(P, LRAMM_K_RFACTOR, s,
          sgemm(0, 0, d.r, l, l, 1.f, at<float>(ws, S.S2T), l, 0, at<float>(ws, S.L1), l, 0.f, at<float>(ws, S.Vj), l,
                s));
    if (m_only_done) *m_only_done = true;
    return LRAMM_OK;
  }
  bool finalized = false;
  TIMED(P, LRAMM_K_SVD, s, launch_jacobi(jb, l, max_sweeps, st, s, &finalized));
  if (!finalized) TIMED(P, LRAMM_K_SVDSORT, s, launch_svd_finalize(fb, l, d.r, s));
  return LRAMM_OK;
}

// The plan's second stream and fork / join events, made on first use on the
// calling thread's current device (remade if the device changes).
lramm_status ensure_streams(lramm_plan_s* P) {
  int dev = 0;
  LRAMM_CUDA_TRY(cudaGetDevice(&dev));
  if (P->s2 && P->dev == dev) return LRAMM_OK;
  if (P->s2) {
    cudaStreamDestroy(P->s2);
    cudaEventDestroy(P->ev_fork);
    cudaEventDestroy(P->ev_join);
    cudaEventDestroy(P->ev_stag);
    P->s2 = nullptr;
  }
  LRAMM_CUDA_TRY(cudaStreamCreateWithFlags(&P->s2, cudaStreamNonBlocking));
  LRAMM_CUDA_TRY(cudaEventCreateWithFlags(&P->ev_fork, cudaEventDisableTiming));
  LRAMM_CUDA_TRY(cudaEventCreateWithFlags(&P->ev_join, cudaEventDisableTiming));
  LRAMM_CUDA_TRY(cudaEventCreateWithFlags(&P->ev_stag, cudaEventDisableTiming));
  P->dev = dev;
  return LRAMM_OK;
}

SideRun side_run(const lramm_plan_s* P, int which, const void* X) {
  const lramm_desc& d = P->d;
  return SideRun{X, which == 0 ? d.lda : d.ldb, (which == 0 ? d.a_type : d.b_type) == LRAMM_BF16,
                 &P->side[which]};
}

// ---------------------------------------------------------------------------
// Range-finder form (the two-stage scheme of Sec. 2.2 applied to the right
// operand W, k x n): Q (k x l) = orth of the sketch W Omega (Philox stream 1)
// after q power iterations, each product re-orthonormalised.  With `keep`
// the chain the backward needs is stored: Q_0..Q_q in bq, Z_1..Z_q in bz and
// the Cholesky factors of orthonormalisation o (o = 0 for Y_0; 2i-1 for
// Y'_i = W^T Q_{i-1}; 2i for Y_i = W Z_i) in bl[o] = {L1, L2}.  On exit Q is
// in the side's R0.
float* bl_slot(lramm_plan_s* P, void* ws, int o, int which) {
  const int64_t l = P->l;
  return at<float>(ws, P->bl) + ((int64_t)o * 2 + which) * l * l;
}

lramm_status range_finder_side(lramm_plan_s* P, const SideRun& sd, void* ws, bool keep, cudaStream_t s) {
  const lramm_desc& d = P->d;
  const int l = P->l;
  const SideLayout& S = *sd.S;
  int* st = at<int>(ws, 0);
  float* R0 = at<float>(ws, S.R0);
  float* R1 = at<float>(ws, S.R1);
  float* C0 = at<float>(ws, S.C0);
  float* C1 = at<float>(ws, S.C1);
  const size_t ll = sizeof(float) * l * l;
  auto keep_L = [&](int o, int passes) -> lramm_status {
    if (!keep) return LRAMM_OK;
    LRAMM_CUDA_TRY(cudaMemcpyAsync(bl_slot(P, ws, o, 0), at<float>(ws, S.L1), ll, cudaMemcpyDeviceToDevice, s));
    if (passes == 2)
      LRAMM_CUDA_TRY(cudaMemcpyAsync(bl_slot(P, ws, o, 1), at<float>(ws, S.L2), ll, cudaMemcpyDeviceToDevice, s));
    return LRAMM_OK;
  };
  float* Om = at<float>(ws, S.omega);
  TIMED(P, LRAMM_K_OMEGA, s, launch_gaussian(d.seed, 1u, S.cols, l, Om, l, s));
  TIMED(P, LRAMM_K_SKETCH, s, x_product(P, ws, *sd.S, 0, sd.X, S.rows, S.cols, sd.ldx, sd.xbf, Om, R0, s));
  const int p0 = d.q > 0 ? 1 : 2;
  float* src[1] = {R0};
  float* tmp[1] = {R1};
  int64_t rows[1] = {S.rows}, cols[1] = {S.cols};
  LRAMM_TRY(orth_sides(P, ws, &sd, 1, src, tmp, src, rows, p0, false, st, s));
  LRAMM_TRY(keep_L(0, p0));
  if (keep)
    LRAMM_CUDA_TRY(cudaMemcpyAsync(at<float>(ws, P->bq), R0, sizeof(float) * S.rows * l, cudaMemcpyDeviceToDevice, s));
  for (int it = 0; it < d.q; ++it) {
    TIMED(P, LRAMM_K_SKETCH, s, x_product(P, ws, *sd.S, 1, sd.X, S.rows, S.cols, sd.ldx, sd.xbf, R0, C0, s));
    float* csrc[1] = {C0};
    float* ctmp[1] = {C1};
    LRAMM_TRY(orth_sides(P, ws, &sd, 1, csrc, ctmp, csrc, cols, 1, false, st, s));
    LRAMM_TRY(keep_L(2 * it + 1, 1));
    if (keep)
      LRAMM_CUDA_TRY(cudaMemcpyAsync(at<float>(ws, P->bz) + (int64_t)it * S.cols * l, C0, sizeof(float) * S.cols * l,
                                     cudaMemcpyDeviceToDevice, s));
    TIMED(P, LRAMM_K_SKETCH, s, x_product(P, ws, *sd.S, 0, sd.X, S.rows, S.cols, sd.ldx, sd.xbf, C0, R0, s));
    const int pi = it == d.q - 1 ? 2 : 1;
    LRAMM_TRY(orth_sides(P, ws, &sd, 1, src, tmp, src, rows, pi, false, st, s));
    LRAMM_TRY(keep_L(2 * it + 2, pi));
    if (keep)
      LRAMM_CUDA_TRY(cudaMemcpyAsync(at<float>(ws, P->bq) + (int64_t)(it + 1) * S.rows * l, R0,
                                     sizeof(float) * S.rows * l, cudaMemcpyDeviceToDevice, s));
  }
  return LRAMM_OK;
}

// C = alpha A B^T + beta C (A: M x K, B: N x K, rows K-contiguous): TF32
// tensor cores when the plan runs its operand products in TF32, FP32 SIMT
// otherwise.
lramm_status nt_product(lramm_plan_s* P, void* ws, int64_t M, int64_t N, int64_t K, float alpha, const float* A,
                        int64_t lda, const float* B, int64_t ldb, float beta, float* C, int64_t ldc, cudaStream_t s) {
  if (P->d.sketch != LRAMM_SKETCH_F32 && tgemm_tc_supported(A, B, lda, ldb, M, N, K))
    return tgemm_tc(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, at<float>(ws, P->qpart), P->qpart_floats,
                    at<int>(ws, 0), s);
  return sgemm(0, 1, M, N, K, alpha, A, lda, 0, B, ldb, beta, C, ldc, s);
}

// Right-multiplication by L^-1 (L lower triangular, l x l): out = X L^-1
// (rows x l), through L^-T = I L^-T (the panel triangular solve on the
// identity) and one product X (L^-T)^T.
lramm_status mul_linv(lramm_plan_s* P, void* ws, const float* L, const float* X, int64_t rows, float* out,
                      cudaStream_t s) {
  const int l = P->l;
  float* I = at<float>(ws, P->tI);
  float* LiT = at<float>(ws, P->tLi);
  LRAMM_TRY(launch_identity(I, l, s));
  SmallBatch tb{};
  tb.n = 1;
  tb.p[0] = SmallProb{I, LiT, L, l};
  LRAMM_TRY(launch_trsm_panel(tb, l, s));
  return nt_product(P, ws, rows, l, l, 1.f, X, l, LiT, l, 0.f, out, l, s);
}

// Adjoint of the thin QR Y = Q R (R = L1^T, or L2^T L1^T after two
// CholeskyQR passes) for a loss that sees Y only through Q:
// dY = (dQ + Q copyltu(M)) R^-T, M = -dQ^T Q; R^-T = L1^-1 or L2^-1 L1^-1.
// dQ (rows x l) is overwritten.
lramm_status qr_adjoint(lramm_plan_s* P, void* ws, const float* Q, int64_t rows, const float* L1, const float* L2,
                        float* dQ, float* dY, cudaStream_t s) {
  const int l = P->l;
  float* M = at<float>(ws, P->tM);
  float* Mc = at<float>(ws, P->tMc);
  LRAMM_TRY(x_product(P, ws, P->side[1], 1, dQ, rows, l, l, 0, Q, M, s));   // M = dQ^T Q
  LRAMM_TRY(launch_copyltu(M, Mc, l, s));
  // dQ += Q copyltu(-M); copyltu(M) is symmetric, so it serves as the N x K operand
  LRAMM_TRY(nt_product(P, ws, rows, l, l, -1.f, Q, l, Mc, l, 1.f, dQ, l, s));
  if (!L2) return mul_linv(P, ws, L1, dQ, rows, dY, s);
  float* T2 = at<float>(ws, P->tY2);
  LRAMM_TRY(mul_linv(P, ws, L2, dQ, rows, T2, s));
  return mul_linv(P, ws, L1, T2, rows, dY, s);
}

// One QM product on codes: the tensor-core kernel (INT8 codes as BF16, INT4 /
// E4M3 codes as FP8; fused dequantisation), the SIMT kernel where the
// operands do not meet its alignment rules.
lramm_status qm_product(lramm_plan_s* P, void* ws, const void* L, const void* R, int64_t M, int64_t N, int64_t K,
                        int64_t ldl, int64_t ldr, int prec, int per_row, const float* sL, const float* sR, float alpha,
                        float beta, const float* C, int64_t ldc, float* D, int64_t ldd, cudaStream_t s) {
  if (qgemm_tc_supported(prec, L, R, ldl, ldr, M, N, K))
    return qgemm_tc(prec, L, R, M, N, K, ldl, ldr, per_row, sL, sR, alpha, beta, C, ldc, D, ldd, at<float>(ws, P->qpart),
                    P->qpart_floats, at<int>(ws, 0), s);
  return qgemm(L, R, M, N, K, ldl, ldr, prec, per_row, sL, sR, alpha, beta, C, ldc, D, ldd, 0, s);
}

// The codes of one QM operand: container (ld = K padded to 32), scales (per
// row or one) and, for MXFP4, block exponents.
struct QOp {
  void* c;
  float* s;
  int8_t* x;
};

lramm_status quant_op(lramm_plan_s* P, void* ws, const float* X, int64_t rows, int64_t cols, int64_t ldx, int prec,
                      const QOp& op, int64_t ldq, cudaStream_t s, bool second_stream = false) {
  if (prec == LRAMM_P_MXFP4) return quantize_mx(X, rows, cols, ldx, static_cast<int8_t*>(op.c), ldq, op.x, s);
  return quantize_rows(X, rows, cols, ldx, prec, P->d.scale == LRAMM_S_ROWCOL, op.c, ldq, op.s,
                       at<unsigned int>(ws, second_stream ? P->amax2 : P->amax), s);
}

// Which factor codes of the chain lramm_matmul forms on the operands' own
// streams, before they join (each factor is quantised as soon as its
// operand's randomized SVD is assembled; the chain then starts from E1).
struct PreQuant {
  bool vw, z, u;
};
PreQuant pre_quant(const lramm_desc& d, bool on) {
  PreQuant q{false, false, false};
  if (!on) return q;
  q.vw = d.prec[0] != LRAMM_P_F32;
  q.z = d.prec[1] != LRAMM_P_F32;
  q.u = d.lead == 0 && d.prec[2] != LRAMM_P_F32 && d.prec[2] != LRAMM_P_MXFP4;
  return q;
}

lramm_status qm_op(lramm_plan_s* P, void* ws, const QOp& L, const QOp& R, int64_t M, int64_t N, int64_t Kq, int prec,
                   float alpha, float beta, const float* C, int64_t ldc, float* D, int64_t ldd, cudaStream_t s) {
  if (prec == LRAMM_P_MXFP4)
    return qgemm_mx(static_cast<const int8_t*>(L.c), L.x, static_cast<const int8_t*>(R.c), R.x, M, N, Kq, Kq, Kq,
                    alpha, beta, C, ldc, D, ldd, s);
  return qm_product(P, ws, L.c, R.c, M, N, Kq, Kq, Kq, prec, P->d.scale == LRAMM_S_ROWCOL, L.s, R.s, alpha, beta, C,
                    ldc, D, ldd, s);
}

// The MXFP4 operands of an E3 term as exact BF16 values (the same decisions
// as quantize_mx), for the tensor-core term product.
lramm_status mx_values(lramm_plan_s* P, void* ws, const float* Ut, const float* E2t, int64_t off, int64_t K,
                       int64_t ldq, cudaStream_t s) {
  const lramm_desc& d = P->d;
  TIMED(P, LRAMM_K_QUANT, s,
        quantize_mx_values(Ut + off, d.m, K, d.r, at<__nv_bfloat16>(ws, P->vU), ldq, s));
  TIMED(P, LRAMM_K_QUANT, s,
        quantize_mx_values(E2t + off, d.n, K, d.r, at<__nv_bfloat16>(ws, P->vE), ldq, s));
  return LRAMM_OK;
}

// E3 with the lead / tail split: the first `lead` rank directions in
// lead_prec with split-precision residuals, the rest in prec[2]; the terms
// accumulate into D (the first one carries beta C).  With an INT8 lead and an
// INT8 or MXFP4 tail every term runs in one tensor-core launch
// (qterms_tc: one pass over D; the MXFP4 tail as exact BF16 values);
// otherwise each term is its own product accumulating into D.
lramm_status e3_lead_tail(lramm_plan_s* P, const float* Ut, const float* E2t, const float* C, float* D, void* ws,
                          cudaStream_t s) {
  const lramm_desc& d = P->d;
  const int64_t r = d.r, lead = d.lead, tail = r - lead, lq = P->lq, tq = round_up(tail > 0 ? tail : 1, 32);
  const int lp = d.lead_prec, per_row = d.scale == LRAMM_S_ROWCOL;
  const bool fused = lp == LRAMM_P_INT8 && (tail == 0 || d.prec[2] == LRAMM_P_INT8 || d.prec[2] == LRAMM_P_MXFP4);
  if (fused) {
    const QOp uh{at<void>(ws, P->cUh), at<float>(ws, P->sUh), nullptr};
    const QOp ul{at<void>(ws, P->cUl), at<float>(ws, P->sUl), nullptr};
    const QOp eh{at<void>(ws, P->cEh), at<float>(ws, P->sEh), nullptr};
    const QOp el{at<void>(ws, P->cEl), at<float>(ws, P->sEl), nullptr};
    float* tres = at<float>(ws, P->tres);
    const void* Lt[4];
    const void* Rt[4];
    int64_t Kt[4], ldl[4], ldr[4];
    const float* sLt[4];
    const float* sRt[4];
    int nt = 0;
    auto add = [&](const void* a, const void* b, int64_t K, int64_t ld, const float* sa, const float* sb) {
      Lt[nt] = a;
      Rt[nt] = b;
      Kt[nt] = K;
      ldl[nt] = ld;
      ldr[nt] = ld;
      sLt[nt] = sa;
      sRt[nt] = sb;
      ++nt;
    };
    TIMED(P, LRAMM_K_QUANT, s, quant_op(P, ws, Ut, d.m, lead, r, lp, uh, lq, s));
    TIMED(P, LRAMM_K_QUANT, s, quant_op(P, ws, E2t, d.n, lead, r, lp, eh, lq, s));
    add(uh.c, eh.c, lq, lq, uh.s, eh.s);
    if (d.lead_split >= 1) {   // + QM(U~_l^lo, E2_l^hi)
      TIMED(P, LRAMM_K_QUANT, s, residual_rows(Ut, d.m, lead, r, lp, uh.c, lq, uh.s, per_row, tres, lead, s));
      TIMED(P, LRAMM_K_QUANT, s, quant_op(P, ws, tres, d.m, lead, lead, lp, ul, lq, s));
      add(ul.c, eh.c, lq, lq, ul.s, eh.s);
    }
    if (d.lead_split >= 2) {   // + QM(U~_l^hi, E2_l^lo)
      TIMED(P, LRAMM_K_QUANT, s, residual_rows(E2t, d.n, lead, r, lp, eh.c, lq, eh.s, per_row, tres, lead, s));
      TIMED(P, LRAMM_K_QUANT, s, quant_op(P, ws, tres, d.n, lead, lead, lp, el, lq, s));
      add(uh.c, el.c, lq, lq, uh.s, el.s);
    }
    if (tail > 0 && d.prec[2] == LRAMM_P_MXFP4) {
      LRAMM_TRY(mx_values(P, ws, Ut, E2t, lead, tail, tq, s));
      add(at<void>(ws, P->vU), at<void>(ws, P->vE), tq, tq, nullptr, nullptr);
    } else if (tail > 0) {
      const QOp ut{at<void>(ws, P->cU), at<float>(ws, P->sU), nullptr};
      const QOp et{at<void>(ws, P->cE2), at<float>(ws, P->sE2), nullptr};
      TIMED(P, LRAMM_K_QUANT, s, quant_op(P, ws, Ut + lead, d.m, tail, r, d.prec[2], ut, tq, s));
      TIMED(P, LRAMM_K_QUANT, s, quant_op(P, ws, E2t + lead, d.n, tail, r, d.prec[2], et, tq, s));
      add(ut.c, et.c, tq, tq, ut.s, et.s);
    }
    if (qterms_tc_supported(nt, Lt, Rt, Kt, ldl, ldr, sLt, d.m, d.n)) {
      TIMED(P, LRAMM_K_E3, s,
            qterms_tc(nt, Lt, Rt, Kt, ldl, ldr, sLt, sRt, per_row, d.m, d.n, d.alpha, d.beta, C, d.ldc, D, d.ldc,
                      at<int>(ws, 0), s));
      return LRAMM_OK;
    }
  }
  const QOp uh{at<void>(ws, P->cUh), at<float>(ws, P->sUh), nullptr};
  const QOp ul{at<void>(ws, P->cUl), at<float>(ws, P->sUl), nullptr};
  const QOp eh{at<void>(ws, P->cEh), at<float>(ws, P->sEh), nullptr};
  const QOp el{at<void>(ws, P->cEl), at<float>(ws, P->sEl), nullptr};
  float* tres = at<float>(ws, P->tres);
  TIMED(P, LRAMM_K_QUANT, s, quant_op(P, ws, Ut, d.m, lead, r, lp, uh, lq, s));
  TIMED(P, LRAMM_K_QUANT, s, quant_op(P, ws, E2t, d.n, lead, r, lp, eh, lq, s));
  TIMED(P, LRAMM_K_E3, s, qm_op(P, ws, uh, eh, d.m, d.n, lq, lp, d.alpha, d.beta, C, d.ldc, D, d.ldc, s));
  if (d.lead_split >= 1) {   // + QM(U~_l^lo, E2_l^hi)
    TIMED(P, LRAMM_K_QUANT, s, residual_rows(Ut, d.m, lead, r, lp, uh.c, lq, uh.s, per_row, tres, lead, s));
    TIMED(P, LRAMM_K_QUANT, s, quant_op(P, ws, tres, d.m, lead, lead, lp, ul, lq, s));
    TIMED(P, LRAMM_K_E3, s, qm_op(P, ws, ul, eh, d.m, d.n, lq, lp, d.alpha, 1.f, D, d.ldc, D, d.ldc, s));
  }
  if (d.lead_split >= 2) {   // + QM(U~_l^hi, E2_l^lo)
    TIMED(P, LRAMM_K_QUANT, s, residual_rows(E2t, d.n, lead, r, lp, eh.c, lq, eh.s, per_row, tres, lead, s));
    TIMED(P, LRAMM_K_QUANT, s, quant_op(P, ws, tres, d.n, lead, lead, lp, el, lq, s));
    TIMED(P, LRAMM_K_E3, s, qm_op(P, ws, uh, el, d.m, d.n, lq, lp, d.alpha, 1.f, D, d.ldc, D, d.ldc, s));
  }
  if (tail > 0) {
    if (d.prec[2] == LRAMM_P_F32) {
      TIMED(P, LRAMM_K_E3, s, sgemm(0, 1, d.m, d.n, tail, d.alpha, Ut + lead, r, 0, E2t + lead, r, 1.f, D, d.ldc, s));
    } else {
      const QOp ut{at<void>(ws, P->cU), at<float>(ws, P->sU), at<int8_t>(ws, P->xU)};
      const QOp et{at<void>(ws, P->cE2), at<float>(ws, P->sE2), at<int8_t>(ws, P->xE2)};
      TIMED(P, LRAMM_K_QUANT, s, quant_op(P, ws, Ut + lead, d.m, tail, r, d.prec[2], ut, tq, s));
      TIMED(P, LRAMM_K_QUANT, s, quant_op(P, ws, E2t + lead, d.n, tail, r, d.prec[2], et, tq, s));
      TIMED(P, LRAMM_K_E3, s, qm_op(P, ws, ut, et, d.m, d.n, tq, d.prec[2], d.alpha, 1.f, D, d.ldc, D, d.ldc, s));
    }
  }
  return LRAMM_OK;
}

lramm_status chain_core(lramm_plan_s* P, const float* Ut, const float* Vt, const float* Wt,
                        const float* Zt, const float* C, float* D, void* ws, cudaStream_t s, bool prequantised = false) {
  const lramm_desc& d = P->d;
  const PreQuant pq = pre_quant(d, prequantised);
  const int64_t r = d.r, kp = P->kp, rp = P->rp;
  float* E1 = at<float>(ws, P->E1);
  float* E2t = at<float>(ws, P->E2t);
  // E1 = QM(V^T W, d1): r x r, K = k
  if (d.prec[0] == LRAMM_P_F32) {
    TIMED(P, LRAMM_K_E1, s, sgemm(0, 1, r, r, d.k, 1.f, Vt, d.k, 0, Wt, d.k, 0.f, E1, r, s));
  } else {
    const QOp v{at<void>(ws, P->cV), at<float>(ws, P->sV), at<int8_t>(ws, P->xV)};
    const QOp w{at<void>(ws, P->cW), at<float>(ws, P->sW), at<int8_t>(ws, P->xW)};
    if (!pq.vw) {
      TIMED(P, LRAMM_K_QUANT, s, quant_op(P, ws, Vt, r, d.k, d.k, d.prec[0], v, kp, s));
      TIMED(P, LRAMM_K_QUANT, s, quant_op(P, ws, Wt, r, d.k, d.k, d.prec[0], w, kp, s));
    }
    TIMED(P, LRAMM_K_E1, s, qm_op(P, ws, v, w, r, r, kp, d.prec[0], 1.f, 0.f, nullptr, 0, E1, r, s));
  }
  // E2 = QM(E1 Z~, d2), computed transposed: E2^T = Z~^T E1^T (n x r, K = r)
  if (d.prec[1] == LRAMM_P_F32) {
    TIMED(P, LRAMM_K_E2, s, sgemm(0, 1, d.n, r, r, 1.f, Zt, r, 0, E1, r, 0.f, E2t, r, s));
  } else {
    const QOp z{at<void>(ws, P->cZ), at<float>(ws, P->sZ), at<int8_t>(ws, P->xZ)};
    const QOp e1{at<void>(ws, P->cE1), at<float>(ws, P->sE1), at<int8_t>(ws, P->xE1)};
    if (!pq.z) TIMED(P, LRAMM_K_QUANT, s, quant_op(P, ws, Zt, d.n, r, r, d.prec[1], z, rp, s));
    TIMED(P, LRAMM_K_QUANT, s, quant_op(P, ws, E1, r, r, r, d.prec[1], e1, rp, s));
    TIMED(P, LRAMM_K_E2, s, qm_op(P, ws, z, e1, d.n, r, rp, d.prec[1], 1.f, 0.f, nullptr, 0, E2t, r, s));
  }
  // E3 = QM(U~ E2, d3); D = alpha E3 + beta C  (m x n, K = r)
  const float beta = d.beta;
  if (beta != 0.f && !C) return LRAMM_ERR_INVALID_ARG;
  if (d.lead > 0) return e3_lead_tail(P, Ut, E2t, C, D, ws, s);
  if (d.prec[2] == LRAMM_P_F32) {
    if (beta != 0.f && C != D)
      LRAMM_CUDA_TRY(cudaMemcpy2DAsync(D, sizeof(float) * d.ldc, C, sizeof(float) * d.ldc,
                                       sizeof(float) * d.n, d.m, cudaMemcpyDeviceToDevice, s));
    TIMED(P, LRAMM_K_E3, s, sgemm(0, 1, d.m, d.n, r, d.alpha, Ut, r, 0, E2t, r, beta, D, d.ldc, s));
  } else {
    if (d.prec[2] == LRAMM_P_MXFP4) {   // exact BF16 values on the tensor cores (one unscaled term)
      LRAMM_TRY(mx_values(P, ws, Ut, E2t, 0, r, rp, s));
      const void* Lt[1] = {at<void>(ws, P->vU)};
      const void* Rt[1] = {at<void>(ws, P->vE)};
      const int64_t Kt[1] = {rp}, ldq[1] = {rp};
      const float* sn[1] = {nullptr};
      if (qterms_tc_supported(1, Lt, Rt, Kt, ldq, ldq, sn, d.m, d.n)) {
        TIMED(P, LRAMM_K_E3, s,
              qterms_tc(1, Lt, Rt, Kt, ldq, ldq, sn, sn, 0, d.m, d.n, d.alpha, beta, C, d.ldc, D, d.ldc,
                        at<int>(ws, 0), s));
        return LRAMM_OK;
      }
    }
    const QOp u{at<void>(ws, P->cU), at<float>(ws, P->sU), at<int8_t>(ws, P->xU)};
    const QOp e2{at<void>(ws, P->cE2), at<float>(ws, P->sE2), at<int8_t>(ws, P->xE2)};
    if (!pq.u) TIMED(P, LRAMM_K_QUANT, s, quant_op(P, ws, Ut, d.m, r, r, d.prec[2], u, rp, s));
    TIMED(P, LRAMM_K_QUANT, s, quant_op(P, ws, E2t, d.n, r, r, d.prec[2], e2, rp, s));
    TIMED(P, LRAMM_K_E3, s, qm_op(P, ws, u, e2, d.m, d.n, rp, d.prec[2], d.alpha, beta, C, d.ldc, D, d.ldc, s));
  }
  return LRAMM_OK;
}

}  // namespace

extern "C" {

const char* lramm_last_cuda_error(void) { return g_cuda_err; }

uint64_t lramm_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

const char* lramm_status_str(lramm_status st) {
  switch (st) {
    case LRAMM_OK: return "ok";
    case LRAMM_ERR_INVALID_ARG: return "invalid argument";
    case LRAMM_ERR_UNSUPPORTED: return "unsupported configuration";
    case LRAMM_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
    case LRAMM_ERR_CUDA: return "CUDA runtime error";
    case LRAMM_ERR_NUMERIC: return "non-positive pivot in Cholesky (rank-deficient sketch)";
    case LRAMM_ERR_TIMEOUT: return "bounded device wait ran out";
    case LRAMM_WARN_NOCONV: return "Jacobi SVD reached its sweep cap";
  }
  return "unknown status";
}

lramm_status lramm_plan_create(const lramm_desc* desc, lramm_plan_t* out) {
  if (!out) return LRAMM_ERR_INVALID_ARG;
  const lramm_status v = validate(desc);
  if (v != LRAMM_OK) return v;
  lramm_plan_s* P = new (std::nothrow) lramm_plan_s();
  if (!P) return LRAMM_ERR_INVALID_ARG;
  P->d = *desc;
  P->timing = (desc->flags & LRAMM_FLAG_TIMING) != 0;
  P->l = desc->r + desc->p;
  layout(P);
  *out = P;
  return LRAMM_OK;
}

lramm_status lramm_plan_destroy(lramm_plan_t plan) {
  if (plan) {
    for (TimerRec& r : plan->recs) {
      cudaEventDestroy(r.a);
      cudaEventDestroy(r.b);
    }
    if (plan->gexec) cudaGraphExecDestroy(plan->gexec);
    if (plan->s2) {
      cudaStreamSynchronize(plan->s2);
      cudaStreamDestroy(plan->s2);
      cudaEventDestroy(plan->ev_fork);
      cudaEventDestroy(plan->ev_join);
      cudaEventDestroy(plan->ev_stag);
    }
  }
  delete plan;
  return LRAMM_OK;
}

lramm_status lramm_timing_read(lramm_plan_t plan, float* ms, int32_t* launches) {
  if (!plan || !ms || !launches || !plan->timing) return LRAMM_ERR_INVALID_ARG;
  for (int k = 0; k < LRAMM_K_COUNT; ++k) {
    ms[k] = 0.f;
    launches[k] = 0;
  }
  for (size_t i = 0; i < plan->used; ++i) {
    const TimerRec& r = plan->recs[i];
    LRAMM_CUDA_TRY(cudaEventSynchronize(r.b));
    float t = 0.f;
    LRAMM_CUDA_TRY(cudaEventElapsedTime(&t, r.a, r.b));
    ms[r.kind] += t;
    launches[r.kind] += 1;
  }
  return LRAMM_OK;
}

const char* lramm_kernel_kind_name(int32_t kind) {
  static const char* names[LRAMM_K_COUNT] = {"omega", "sketch", "gram", "chol", "trsm", "rfactor", "svd",
                                             "svdsort", "assemble", "quant", "e1", "e2", "e3", "other",
                                             "backward", "qr_adjoint", "reconstruct"};
  return (kind >= 0 && kind < LRAMM_K_COUNT) ? names[kind] : "unknown";
}

lramm_status lramm_workspace_size(lramm_plan_t plan, size_t* bytes) {
  if (!plan || !bytes) return LRAMM_ERR_INVALID_ARG;
  *bytes = plan->total;
  return LRAMM_OK;
}

lramm_status lramm_rsvd(lramm_plan_t plan, int32_t which, const void* X, float* U, float* S, float* V,
                        void* ws, size_t ws_bytes, void* stream) {
  if (!plan || (which != 0 && which != 1) || !X || !U || !S || !V) return LRAMM_ERR_INVALID_ARG;
  if (plan->l > svd_max_l()) return LRAMM_ERR_UNSUPPORTED;
  LRAMM_TRY(check_ws(plan, ws, ws_bytes));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const SideLayout& Sd = plan->side[which];
  const int l = plan->l, r = plan->d.r;
  plan->used = 0;
  LRAMM_CUDA_TRY(cudaMemsetAsync(ws, 0, kStatusWords * sizeof(int), s));
  const SideRun sd = side_run(plan, which, X);
  const int zero[1] = {0};
  LRAMM_TRY(rsvd_sides(plan, &sd, &which, 1, ws, zero, zero, s));
  TIMED(plan, LRAMM_K_ASSEMBLE, s,
        assemble(plan, ws, Sd, Sd.rows, r, at<float>(ws, Sd.R0), at<float>(ws, Sd.S1T), U, r, 0,
                 at<float>(ws, Sd.R0), l, 0, at<float>(ws, Sd.S1), r, s));
  TIMED(plan, LRAMM_K_ASSEMBLE, s,
        assemble(plan, ws, Sd, Sd.cols, r, at<float>(ws, Sd.C0), at<float>(ws, Sd.S2T), V, r, 0,
                 at<float>(ws, Sd.C0), l, 0, at<float>(ws, Sd.S2), r, s));
  LRAMM_CUDA_TRY(cudaMemcpyAsync(S, at<float>(ws, Sd.sig), sizeof(float) * r, cudaMemcpyDeviceToDevice, s));
  return LRAMM_OK;
}

// ---- Algorithm 4: quantised SVD of one operand ---------------------------

namespace {

bool qsvd_prec_ok(int p) { return p == LRAMM_P_INT8 || p == LRAMM_P_INT4 || p == LRAMM_P_E4M3; }

// Workspace beyond the plan's: the BF16 copy of INT4 codes that meet INT8
// codes in one product, and the split-K partials of that product.
struct QsvdLayout {
  int pp;         // precision of the code product; -1: the pair has none (INT8 / E4M3)
  int conv_side;  // 0: U codes, 1: V codes are rewritten as BF16; -1: none
  int64_t kq;     // K of the product: r rounded up to 32 (the codes are zero beyond r)
  size_t conv, part, part_floats, total;
};

QsvdLayout qsvd_layout(const lramm_plan_s* P, int which, int pu, int pv) {
  QsvdLayout L{};
  const SideLayout& S = P->side[which];
  L.kq = round_up(P->d.r, 32);
  L.conv_side = -1;
  if (pu == pv) {
    L.pp = pu;
  } else if (pu != LRAMM_P_INT8 && pv != LRAMM_P_INT8) {
    L.pp = LRAMM_P_E4M3;   // INT4 and E4M3 codes are both e4m3 bytes
  } else if (pu == LRAMM_P_INT4 || pv == LRAMM_P_INT4) {
    L.pp = LRAMM_P_INT8;   // INT4 codes as BF16 values beside INT8 codes: exact sums
    L.conv_side = pu == LRAMM_P_INT4 ? 0 : 1;
  } else {
    L.pp = -1;
  }
  size_t off = static_cast<size_t>(round_up(static_cast<int64_t>(P->total), kAlign));
  L.conv = off;
  if (L.conv_side >= 0)
    off += static_cast<size_t>(round_up(2 * (L.conv_side == 0 ? S.rows : S.cols) * L.kq, kAlign));
  L.part = off;
  L.part_floats = L.pp >= 0 ? qgemm_tc_part_floats(L.pp, S.rows, S.cols, L.kq) : 0;
  off += static_cast<size_t>(round_up(static_cast<int64_t>(sizeof(float) * std::max<size_t>(L.part_floats, 4)), kAlign));
  L.total = off;
  return L;
}

}  // namespace

size_t lramm_qsvd_ws_bytes(lramm_plan_t plan, int32_t which, int32_t prec_u, int32_t prec_v) {
  if (!plan || (which != 0 && which != 1) || !qsvd_prec_ok(prec_u) || !qsvd_prec_ok(prec_v)) return 0;
  return qsvd_layout(plan, which, prec_u, prec_v).total;
}

lramm_status lramm_qsvd(lramm_plan_t plan, int32_t which, const void* X, int32_t prec_u, int32_t prec_v, void* Uc,
                        float* Us, void* Vc, float* Vs, int64_t ldq, float* Uf, float* Vf, float* Xr, int64_t ldxr,
                        void* ws, size_t ws_bytes, void* stream) {
  if (!plan || (which != 0 && which != 1) || !X || !Uc || !Us || !Vc || !Vs) return LRAMM_ERR_INVALID_ARG;
  if (prec_u == LRAMM_P_MXFP4 || prec_v == LRAMM_P_MXFP4) return LRAMM_ERR_UNSUPPORTED;
  if (!qsvd_prec_ok(prec_u) || !qsvd_prec_ok(prec_v)) return LRAMM_ERR_INVALID_ARG;
  const lramm_desc& d = plan->d;
  const SideLayout& Sd = plan->side[which];
  const int l = plan->l, r = d.r;
  if (ldq < r || ldq % 32 != 0) return LRAMM_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(Uc) % 16 || reinterpret_cast<uintptr_t>(Vc) % 16) return LRAMM_ERR_INVALID_ARG;
  if (Xr && ldxr < Sd.cols) return LRAMM_ERR_INVALID_ARG;
  if (plan->l > svd_max_l()) return LRAMM_ERR_UNSUPPORTED;
  const QsvdLayout Q = qsvd_layout(plan, which, prec_u, prec_v);
  if (Xr && Q.pp < 0) return LRAMM_ERR_UNSUPPORTED;
  if (!ws || ws_bytes < Q.total || reinterpret_cast<uintptr_t>(ws) % kAlign) return LRAMM_ERR_WORKSPACE;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int per_row = d.scale == LRAMM_S_ROWCOL;
  plan->used = 0;
  LRAMM_CUDA_TRY(cudaMemsetAsync(ws, 0, kStatusWords * sizeof(int), s));
  // SVD(A, k) and U~ = U_k Sigma_k: the small SVD's left vectors carry sigma
  const SideRun sd = side_run(plan, which, X);
  const int one[1] = {1}, zero[1] = {0};
  LRAMM_TRY(rsvd_sides(plan, &sd, &which, 1, ws, one, zero, s));
  // the factors: caller's buffers when given, else the plan's factor buffers
  // (A side: U~ m x r in U~'s, V k x r in V^T's; B side: U~ k x r in W^T's,
  // V n x r in Z~^T's -- each at least as large)
  float* Ut = Uf ? Uf : at<float>(ws, which == 0 ? plan->Ut : plan->Wt);
  float* V = Vf ? Vf : at<float>(ws, which == 0 ? plan->Vt : plan->Zt);
  TIMED(plan, LRAMM_K_ASSEMBLE, s,
        assemble(plan, ws, Sd, Sd.rows, r, at<float>(ws, Sd.R0), at<float>(ws, Sd.S1T), Ut, r, 0,
                 at<float>(ws, Sd.R0), l, 0, at<float>(ws, Sd.S1), r, s));
  TIMED(plan, LRAMM_K_ASSEMBLE, s,
        assemble(plan, ws, Sd, Sd.cols, r, at<float>(ws, Sd.C0), at<float>(ws, Sd.S2T), V, r, 0,
                 at<float>(ws, Sd.C0), l, 0, at<float>(ws, Sd.S2), r, s));
  unsigned int* amax = at<unsigned int>(ws, plan->amax);
  TIMED(plan, LRAMM_K_QUANT, s, quantize_rows(Ut, Sd.rows, r, r, prec_u, per_row, Uc, ldq, Us, amax, s));
  TIMED(plan, LRAMM_K_QUANT, s, quantize_rows(V, Sd.cols, r, r, prec_v, per_row, Vc, ldq, Vs, amax, s));
  if (!Xr) return LRAMM_OK;
  const void* L = Uc;
  const void* R = Vc;
  int64_t ldl = ldq, ldr = ldq;
  if (Q.conv_side >= 0) {
    void* cv = at<void>(ws, Q.conv);
    const int64_t rows = Q.conv_side == 0 ? Sd.rows : Sd.cols;
    TIMED(plan, LRAMM_K_RECON, s, fp8_codes_to_bf16(Q.conv_side == 0 ? Uc : Vc, rows, Q.kq, ldq, cv, Q.kq, s));
    if (Q.conv_side == 0) {
      L = cv;
      ldl = Q.kq;
    } else {
      R = cv;
      ldr = Q.kq;
    }
  }
  TIMED(plan, LRAMM_K_RECON, s,
        qgemm_tc(Q.pp, L, R, Sd.rows, Sd.cols, Q.kq, ldl, ldr, per_row, Us, Vs, 1.f, 0.f, nullptr, 0, Xr, ldxr,
                 at<float>(ws, Q.part), Q.part_floats, at<int>(ws, 0), s));
  return LRAMM_OK;
}

lramm_status lramm_chain(lramm_plan_t plan, const float* Ut, const float* Vt, const float* Wt,
                         const float* Zt, const float* C, float* D, void* ws, size_t ws_bytes,
                         void* stream) {
  if (!plan || !Ut || !Vt || !Wt || !Zt || !D) return LRAMM_ERR_INVALID_ARG;
  LRAMM_TRY(check_ws(plan, ws, ws_bytes));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  plan->used = 0;
  LRAMM_CUDA_TRY(cudaMemsetAsync(ws, 0, kStatusWords * sizeof(int), s));
  return chain_core(plan, Ut, Vt, Wt, Zt, C, D, ws, s);
}

lramm_status matmul_body(lramm_plan_t plan, const void* A, const void* B, const float* C, float* D, void* ws,
                         cudaStream_t s);

lramm_status lramm_matmul(lramm_plan_t plan, const void* A, const void* B, const float* C, float* D,
                          void* ws, size_t ws_bytes, void* stream) {
  if (!plan || !A || !B || !D) return LRAMM_ERR_INVALID_ARG;
  if (plan->d.beta != 0.f && !C) return LRAMM_ERR_INVALID_ARG;
  if (plan->l > svd_max_l()) return LRAMM_ERR_UNSUPPORTED;
  LRAMM_TRY(check_ws(plan, ws, ws_bytes));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (!(plan->d.flags & LRAMM_FLAG_GRAPH) || plan->timing || s == nullptr) return matmul_body(plan, A, B, C, D, ws, s);
  // CUDA graph: replay the captured call when the arguments match, else capture anew
  int dev = 0;
  LRAMM_CUDA_TRY(cudaGetDevice(&dev));
  const void* key[6] = {A, B, C, D, ws, stream};
  bool same = plan->gexec && plan->gdev == dev;
  for (int i = 0; i < 6 && same; ++i) same = plan->gkey[i] == key[i];
  if (!same) {
    if (plan->gexec) {
      cudaGraphExecDestroy(plan->gexec);
      plan->gexec = nullptr;
    }
    LRAMM_TRY(ensure_streams(plan));   // made outside the capture
    LRAMM_CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    const unsigned long long n0 = g_launches.load(std::memory_order_relaxed);
    const lramm_status st = matmul_body(plan, A, B, C, D, ws, s);
    plan->glaunches = g_launches.load(std::memory_order_relaxed) - n0;
    g_launches.fetch_sub(plan->glaunches, std::memory_order_relaxed);   // captured, not launched
    cudaGraph_t g = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(s, &g);
    if (st != LRAMM_OK || ce != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      if (st != LRAMM_OK) return st;
      LRAMM_CUDA_TRY(ce);
    }
    const cudaError_t ie = cudaGraphInstantiate(&plan->gexec, g, 0);
    cudaGraphDestroy(g);
    LRAMM_CUDA_TRY(ie);
    for (int i = 0; i < 6; ++i) plan->gkey[i] = key[i];
    plan->gdev = dev;
  }
  // the library's launches inside the graph count as launched on every replay
  for (size_t i = 0; i < plan->glaunches; ++i) count_launch();
  LRAMM_CUDA_TRY(cudaGraphLaunch(plan->gexec, s));
  return LRAMM_OK;
}

lramm_status matmul_body(lramm_plan_t plan, const void* A, const void* B, const float* C, float* D, void* ws,
                         cudaStream_t s) {
  const lramm_desc& d = plan->d;
  const int l = plan->l, r = d.r;
  plan->used = 0;
  LRAMM_CUDA_TRY(cudaMemsetAsync(ws, 0, kStatusWords * sizeof(int), s));
  float* Ut = at<float>(ws, plan->Ut);
  float* Vt = at<float>(ws, plan->Vt);
  float* Wt = at<float>(ws, plan->Wt);
  float* Zt = at<float>(ws, plan->Zt);
  // A: U~ = Q_A (U_s Sigma) (m x r);  V^T = V_s^T P_A^T (r x k)  (M-only
  // form: V^T = Y^T P1^T)
  const SideLayout& SA = plan->side[0];
  const SideLayout& SB = plan->side[1];
  const SideRun sd[2] = {side_run(plan, 0, A), side_run(plan, 1, B)};
  const int which[2] = {0, 1}, s1s[2] = {1, 0}, s2s[2] = {0, 1};
  // Loose Jacobi stopping rule where every term of E3 carries 8-bit-or-less
  // codes: a quantised E3 without lead / tail split, or a lead / tail split
  // whose E1 and E2 are quantised (E2's own code noise then bounds the
  // lead's precision).
  const bool coded_lead = d.lead > 0 && d.prec[0] != LRAMM_P_F32 && d.prec[1] != LRAMM_P_F32;
  const float stopq = ((d.prec[2] != LRAMM_P_F32 && d.lead == 0) || coded_lead) ? kJacobiQuadQuantised : kJacobiQuad;
  // Quantised chains take the M-only small SVD (right factors P1 (R1 U_s
  // Sigma^-1)): their codes see the factors only through the rank-r
  // products, which the two forms give alike up to the Jacobi's leftover,
  // below the codes' noise.  FP32 chains keep V_s.
  const bool m_only = d.prec[2] != LRAMM_P_F32 || d.lead > 0;
  // The two operands' RSVDs are independent: A on the caller's stream, B on
  // the plan's second stream, so that one operand's latency-bound small
  // algebra (a few CTAs) runs beside the other's HBM-bound products.
  LRAMM_TRY(ensure_streams(plan));
  cudaStream_t s2 = plan->s2;
  LRAMM_CUDA_TRY(cudaEventRecord(plan->ev_fork, s));
  LRAMM_CUDA_TRY(cudaStreamWaitEvent(s2, plan->ev_fork, 0));
  // each operand's factors are quantised on its own stream once assembled,
  // so that the first operand's codes form while the second's randomized SVD
  // still runs (the per-tensor amax word of the second stream is its own)
  const PreQuant pq = pre_quant(d, true);
  const QOp qv{at<void>(ws, plan->cV), at<float>(ws, plan->sV), at<int8_t>(ws, plan->xV)};
  const QOp qw{at<void>(ws, plan->cW), at<float>(ws, plan->sW), at<int8_t>(ws, plan->xW)};
  const QOp qz{at<void>(ws, plan->cZ), at<float>(ws, plan->sZ), at<int8_t>(ws, plan->xZ)};
  const QOp qu{at<void>(ws, plan->cU), at<float>(ws, plan->sU), at<int8_t>(ws, plan->xU)};
  auto side_a = [&]() -> lramm_status {
    bool mo = false;
    LRAMM_TRY(rsvd_sides(plan, &sd[0], &which[0], 1, ws, &s1s[0], &s2s[0], s, stopq, m_only, &mo, plan->ev_stag));
    TIMED(plan, LRAMM_K_ASSEMBLE, s,
          assemble(plan, ws, SA, d.m, r, at<float>(ws, SA.R0), at<float>(ws, SA.S1T), Ut, r, 0,
                   at<float>(ws, SA.R0), l, 0, at<float>(ws, SA.S1), r, s, true));
    if (mo)  // V^T = Y^T P1^T
      TIMED(plan, LRAMM_K_ASSEMBLE, s,
            assemble(plan, ws, SA, r, d.k, at<float>(ws, SA.Vj), at<float>(ws, SA.C1), Vt, d.k, 0,
                     at<float>(ws, SA.Vj), l, 1, at<float>(ws, SA.C1), l, s, true));
    else
      TIMED(plan, LRAMM_K_ASSEMBLE, s,
            assemble(plan, ws, SA, r, d.k, at<float>(ws, SA.S2T), at<float>(ws, SA.C0), Vt, d.k, 1,
                     at<float>(ws, SA.S2), r, 1, at<float>(ws, SA.C0), l, s, true));
    if (pq.vw) TIMED(plan, LRAMM_K_QUANT, s, quant_op(plan, ws, Vt, r, d.k, d.k, d.prec[0], qv, plan->kp, s));
    if (pq.u) TIMED(plan, LRAMM_K_QUANT, s, quant_op(plan, ws, Ut, d.m, r, r, d.prec[2], qu, plan->rp, s));
    return LRAMM_OK;
  };
  // B: W^T = U_s^T Q_B^T (r x k);  Z~^T = P_B (V_s Gamma) (n x r)  (M-only
  // form: Z~^T = P1 Y)
  auto side_b = [&]() -> lramm_status {
    bool mo = false;
    LRAMM_TRY(rsvd_sides(plan, &sd[1], &which[1], 1, ws, &s1s[1], &s2s[1], s2, stopq, m_only, &mo, nullptr,
                         plan->ev_stag));
    TIMED(plan, LRAMM_K_ASSEMBLE, s2,
          assemble(plan, ws, SB, r, d.k, at<float>(ws, SB.S1T), at<float>(ws, SB.R0), Wt, d.k, 1,
                   at<float>(ws, SB.S1), r, 1, at<float>(ws, SB.R0), l, s2, true));
    if (mo)  // Z~^T = P1 Y
      TIMED(plan, LRAMM_K_ASSEMBLE, s2,
            assemble(plan, ws, SB, d.n, r, at<float>(ws, SB.C1), at<float>(ws, SB.Vj), Zt, r, 0,
                     at<float>(ws, SB.C1), l, 1, at<float>(ws, SB.Vj), l, s2, true));
    else
      TIMED(plan, LRAMM_K_ASSEMBLE, s2,
            assemble(plan, ws, SB, d.n, r, at<float>(ws, SB.C0), at<float>(ws, SB.S2T), Zt, r, 0,
                     at<float>(ws, SB.C0), l, 0, at<float>(ws, SB.S2), r, s2, true));
    if (pq.vw)
      TIMED(plan, LRAMM_K_QUANT, s2, quant_op(plan, ws, Wt, r, d.k, d.k, d.prec[0], qw, plan->kp, s2, true));
    if (pq.z) TIMED(plan, LRAMM_K_QUANT, s2, quant_op(plan, ws, Zt, d.n, r, r, d.prec[1], qz, plan->rp, s2, true));
    return LRAMM_OK;
  };
  const lramm_status st_a = side_a();
  const lramm_status st_b = side_b();
  // join (also after an error: nothing of this call may still run on s2 once it returns to s's order)
  LRAMM_CUDA_TRY(cudaEventRecord(plan->ev_join, s2));
  LRAMM_CUDA_TRY(cudaStreamWaitEvent(s, plan->ev_join, 0));
  LRAMM_TRY(st_a);
  LRAMM_TRY(st_b);
  return chain_core(plan, Ut, Vt, Wt, Zt, C, D, ws, s, true);
}

lramm_status lramm_info_read(const void* ws, int32_t* info, int32_t n, void* stream) {
  if (!ws || !info || n < 1 || n > 64) return LRAMM_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  LRAMM_CUDA_TRY(cudaMemcpyAsync(info, ws, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s));
  LRAMM_CUDA_TRY(cudaStreamSynchronize(s));
  return LRAMM_OK;
}

lramm_status lramm_status_read(const void* ws, void* stream) {
  if (!ws) return LRAMM_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int h = 0;
  LRAMM_CUDA_TRY(cudaMemcpyAsync(&h, ws, sizeof(int), cudaMemcpyDeviceToHost, s));
  LRAMM_CUDA_TRY(cudaStreamSynchronize(s));
  LRAMM_CUDA_TRY(cudaMemsetAsync(const_cast<void*>(ws), 0, sizeof(int), s));
  return static_cast<lramm_status>(h);
}

lramm_status lramm_philox_words(uint64_t seed, uint32_t stream_id, int64_t n_blocks, uint32_t* out,
                                void* stream) {
  if (n_blocks < 0 || (n_blocks > 0 && !out)) return LRAMM_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(out) % 16) return LRAMM_ERR_INVALID_ARG;
  return launch_philox_words(seed, stream_id, n_blocks, out, static_cast<cudaStream_t>(stream));
}

lramm_status lramm_gaussian(uint64_t seed, uint32_t stream_id, int64_t rows, int64_t cols, float* out,
                            void* stream) {
  if (rows < 0 || cols < 0 || (rows * cols > 0 && !out)) return LRAMM_ERR_INVALID_ARG;
  return launch_gaussian(seed, stream_id, rows, cols, out, cols, static_cast<cudaStream_t>(stream));
}

size_t lramm_quant_ws_bytes(void) { return kAlign; }

size_t lramm_sketch_ws_bytes(int64_t rows, int64_t cols, int64_t l) {
  if (l < 1 || rows < 1 || cols < 1) return 0;
  return kAlign + sizeof(float) * sketch_tc_part_floats((int)l) + sketch_bf_split_bytes(std::max(rows, cols), (int)l);
}

lramm_status lramm_sketch_product(const void* X, int64_t rows, int64_t cols, int64_t ldx, int32_t x_type,
                                  int32_t transpose, const float* B, int64_t l, float* out, int32_t sketch,
                                  void* ws, size_t ws_bytes, void* stream) {
  if (rows < 1 || cols < 1 || ldx < cols || l < 1 || l > 4096 || !X || !B || !out) return LRAMM_ERR_INVALID_ARG;
  if ((x_type != LRAMM_F32 && x_type != LRAMM_BF16) || (transpose != 0 && transpose != 1)) return LRAMM_ERR_INVALID_ARG;
  if (sketch < LRAMM_SKETCH_F32 || sketch > LRAMM_SKETCH_BF16) return LRAMM_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int xbf = x_type == LRAMM_BF16;
  if (sketch != LRAMM_SKETCH_F32) {
    if (!ws || ws_bytes < lramm_sketch_ws_bytes(rows, cols, l) || reinterpret_cast<uintptr_t>(ws) % kAlign)
      return LRAMM_ERR_WORKSPACE;
    float* part = at<float>(ws, kAlign);
    const size_t pf = sketch_tc_part_floats((int)l);
    if (xbf) {
      if (!sketch_bf_supported(ldx, (int)l, X, B)) return LRAMM_ERR_UNSUPPORTED;
      void* split = at<void>(ws, kAlign + sizeof(float) * pf);
      return sketch_bf(transpose, X, rows, cols, ldx, B, (int)l, sketch == LRAMM_SKETCH_TF32 ? 2 : 1, out, part, pf,
                       split, sketch_bf_split_bytes(std::max(rows, cols), (int)l), at<int>(ws, 0), s);
    }
    if (!sketch_tc_supported(xbf, ldx, (int)l, X, B)) return LRAMM_ERR_UNSUPPORTED;
    return sketch_tc(transpose, X, rows, cols, ldx, xbf, B, (int)l, out, part, pf, at<int>(ws, 0), s);
  }
  if (transpose) return sgemm(1, 0, cols, l, rows, 1.f, X, ldx, xbf, B, l, 0.f, out, l, s);
  return sgemm(0, 0, rows, l, cols, 1.f, X, ldx, xbf, B, l, 0.f, out, l, s);
}

lramm_status lramm_quantize(const float* X, int64_t rows, int64_t cols, int64_t ldx, int32_t prec,
                            int32_t per_row, void* codes, int64_t ldcodes, float* scales, void* ws,
                            void* stream) {
  if (rows < 0 || cols < 0 || ldx < cols || ldcodes < cols) return LRAMM_ERR_INVALID_ARG;
  if (prec == LRAMM_P_F32 || !valid_prec(prec)) return LRAMM_ERR_INVALID_ARG;
  if (rows > 0 && (!X || !codes || !scales)) return LRAMM_ERR_INVALID_ARG;
  if (!per_row && rows > 0 && !ws) return LRAMM_ERR_INVALID_ARG;
  return quantize_rows(X, rows, cols, ldx, prec, per_row, codes, ldcodes, scales,
                       static_cast<unsigned int*>(ws), static_cast<cudaStream_t>(stream));
}

lramm_status lramm_quantize_noalloc(const float* X, int64_t rows, int64_t cols, int64_t ldx, int32_t prec,
                                    int32_t per_row, void* codes, int64_t ldcodes, float* scales,
                                    void* stream) {
  if (rows < 0 || cols < 0 || ldx < cols || ldcodes < cols) return LRAMM_ERR_INVALID_ARG;
  if (prec == LRAMM_P_F32 || !valid_prec(prec)) return LRAMM_ERR_INVALID_ARG;
  if (rows > 0 && (!X || !codes || !scales)) return LRAMM_ERR_INVALID_ARG;
  return quantize_rows_noalloc(X, rows, cols, ldx, prec, per_row, codes, ldcodes, scales,
                               static_cast<cudaStream_t>(stream));
}

size_t lramm_noalloc_scratch_bytes(void) { return noalloc_scratch_bytes(); }

lramm_status lramm_quantize_cols(const float* X, int64_t rows, int64_t cols, int64_t ldx, int32_t prec, void* codesT,
                                 int64_t ldcodes, float* scales, void* ws, void* stream) {
  if (!X || !codesT || !scales || !ws || rows < 1 || cols < 1 || ldx < cols || ldcodes < rows) return LRAMM_ERR_INVALID_ARG;
  if (prec != LRAMM_P_INT8 && prec != LRAMM_P_INT4 && prec != LRAMM_P_E4M3) return LRAMM_ERR_INVALID_ARG;
  return quantize_cols2d(X, rows, cols, ldx, prec, codesT, ldcodes, scales, static_cast<unsigned int*>(ws),
                         static_cast<cudaStream_t>(stream));
}

lramm_status lramm_qgemm(const void* L, const void* Rt, int64_t M, int64_t N, int64_t K, int64_t ldl,
                         int64_t ldr, int32_t prec, int32_t per_row, const float* sL, const float* sR,
                         float alpha, float beta, const float* C, int64_t ldc, void* D, int64_t ldd,
                         int32_t out_kind, void* stream) {
  if (M < 0 || N < 0 || K < 0 || K % 16 || ldl < K || ldr < K || ldd < N) return LRAMM_ERR_INVALID_ARG;
  if (prec == LRAMM_P_F32 || !valid_prec(prec)) return LRAMM_ERR_INVALID_ARG;
  if (out_kind != 0 && out_kind != 1) return LRAMM_ERR_INVALID_ARG;
  if (M > 0 && N > 0 && (!L || !Rt || !D)) return LRAMM_ERR_INVALID_ARG;
  if (out_kind == 0 && (!sL || !sR || (beta != 0.f && (!C || ldc < N)))) return LRAMM_ERR_INVALID_ARG;
  return qgemm(L, Rt, M, N, K, ldl, ldr, prec, per_row, sL, sR, alpha, beta, C, ldc, D, ldd, out_kind,
               static_cast<cudaStream_t>(stream));
}

lramm_status lramm_rf_forward(lramm_plan_t plan, const void* X, const void* W, float* C, void* ws, size_t ws_bytes,
                              void* stream) {
  if (!plan || !X || !W || !C) return LRAMM_ERR_INVALID_ARG;
  if (plan->d.sketch == LRAMM_SKETCH_E4M3) return LRAMM_ERR_UNSUPPORTED;
  LRAMM_TRY(check_ws(plan, ws, ws_bytes));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const lramm_desc& d = plan->d;
  const int l = plan->l;
  plan->used = 0;
  LRAMM_CUDA_TRY(cudaMemsetAsync(ws, 0, kStatusWords * sizeof(int), s));
  const SideRun sx = side_run(plan, 0, X), sw = side_run(plan, 1, W);
  LRAMM_TRY(range_finder_side(plan, sw, ws, false, s));
  const float* Q = at<float>(ws, sw.S->R0);
  float* T = at<float>(ws, sx.S->R0);   // m x l
  float* Pt = at<float>(ws, sw.S->C0);  // n x l = (Q^T W)^T
  TIMED(plan, LRAMM_K_SKETCH, s, x_product(plan, ws, *sx.S, 0, X, d.m, d.k, d.lda, sx.xbf, Q, T, s));
  TIMED(plan, LRAMM_K_SKETCH, s, x_product(plan, ws, *sw.S, 1, W, d.k, d.n, d.ldb, sw.xbf, Q, Pt, s));
  if (d.prec[2] == LRAMM_P_F32) {
    TIMED(plan, LRAMM_K_E3, s, nt_product(plan, ws, d.m, d.n, l, d.alpha, T, l, Pt, l, d.beta, C, d.ldc, s));
    return LRAMM_OK;
  }
  const QOp ct{at<void>(ws, plan->cT), at<float>(ws, plan->sT), at<int8_t>(ws, plan->xT)};
  const QOp cp{at<void>(ws, plan->cP), at<float>(ws, plan->sP), at<int8_t>(ws, plan->xP)};
  TIMED(plan, LRAMM_K_QUANT, s, quant_op(plan, ws, T, d.m, l, l, d.prec[2], ct, plan->lp, s));
  TIMED(plan, LRAMM_K_QUANT, s, quant_op(plan, ws, Pt, d.n, l, l, d.prec[2], cp, plan->lp, s));
  TIMED(plan, LRAMM_K_E3, s, qm_op(plan, ws, ct, cp, d.m, d.n, plan->lp, d.prec[2], d.alpha, d.beta, C, d.ldc, C,
                                  d.ldc, s));
  return LRAMM_OK;
}

lramm_status lramm_rf_backward(lramm_plan_t plan, const void* X, const void* W, const float* G, float* dX,
                               float* dW, void* ws, size_t ws_bytes, void* stream) {
  if (!plan || !X || !W || !G || !dX || !dW) return LRAMM_ERR_INVALID_ARG;
  const lramm_desc& d = plan->d;
  if (d.b_type != LRAMM_F32 || d.sketch == LRAMM_SKETCH_E4M3) return LRAMM_ERR_UNSUPPORTED;
  LRAMM_TRY(check_ws(plan, ws, ws_bytes));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int l = plan->l;
  const int64_t m = d.m, n = d.n, k = d.k;
  plan->used = 0;
  LRAMM_CUDA_TRY(cudaMemsetAsync(ws, 0, kStatusWords * sizeof(int), s));
  const SideRun sx = side_run(plan, 0, X), sw = side_run(plan, 1, W);
  LRAMM_TRY(range_finder_side(plan, sw, ws, true, s));
  auto Qi = [&](int i) { return at<float>(ws, plan->bq) + (int64_t)i * k * l; };
  auto Zi = [&](int i) { return at<float>(ws, plan->bz) + (int64_t)(i - 1) * n * l; };
  const float* Q = Qi(d.q);
  float* T = at<float>(ws, sx.S->R0);   // m x l
  float* Pt = at<float>(ws, sw.S->C0);  // n x l
  float* dT = at<float>(ws, plan->tdT);
  float* dPt = at<float>(ws, plan->tdP);
  float* dQ = at<float>(ws, plan->tdQ);
  float* dZ = at<float>(ws, plan->tdZ);
  float* dY = at<float>(ws, plan->tY);
  TIMED(plan, LRAMM_K_SKETCH, s, x_product(plan, ws, *sx.S, 0, X, m, k, d.lda, sx.xbf, Q, T, s));
  TIMED(plan, LRAMM_K_SKETCH, s, x_product(plan, ws, *sw.S, 1, W, k, n, d.ldb, sw.xbf, Q, Pt, s));
  // dT = alpha G P^T (m x l), dP^T = alpha G^T T (n x l)
  TIMED(plan, LRAMM_K_SKETCH, s, x_product(plan, ws, *sw.S, 0, G, m, n, d.ldc, 0, Pt, dT, s));
  TIMED(plan, LRAMM_K_SKETCH, s, x_product(plan, ws, *sw.S, 1, G, m, n, d.ldc, 0, T, dPt, s));
  TIMED(plan, LRAMM_K_BWD, s, launch_scale(dT, m * l, d.alpha, s));
  TIMED(plan, LRAMM_K_BWD, s, launch_scale(dPt, n * l, d.alpha, s));
  // dX = dT Q^T (m x k);  dW = Q dP (k x n)
  TIMED(plan, LRAMM_K_BWD, s, nt_product(plan, ws, m, k, l, 1.f, dT, l, Q, l, 0.f, dX, k, s));
  TIMED(plan, LRAMM_K_BWD, s, nt_product(plan, ws, k, n, l, 1.f, Q, l, dPt, l, 0.f, dW, n, s));
  // dQ = X^T dT + W dP^T (k x l)
  TIMED(plan, LRAMM_K_SKETCH, s, x_product(plan, ws, *sx.S, 1, X, m, k, d.lda, sx.xbf, dT, dQ, s));
  float* tmp = at<float>(ws, plan->tB);
  TIMED(plan, LRAMM_K_SKETCH, s, x_product(plan, ws, *sw.S, 0, W, k, n, d.ldb, sw.xbf, dPt, tmp, s));
  TIMED(plan, LRAMM_K_BWD, s, launch_axpy(dQ, tmp, k * l, 1.f, s));
  // back through the power iterations (Omega fixed)
  for (int i = d.q; i >= 1; --i) {
    const int o = 2 * i;                 // Y_i = W Z_i, Q_i = orth(Y_i)
    const bool two = i == d.q;           // the last basis took two CholeskyQR passes
    TIMED(plan, LRAMM_K_ADJOINT, s,
          qr_adjoint(plan, ws, Qi(i), k, bl_slot(plan, ws, o, 0), two ? bl_slot(plan, ws, o, 1) : nullptr, dQ, dY, s));
    TIMED(plan, LRAMM_K_BWD, s, nt_product(plan, ws, k, n, l, 1.f, dY, l, Zi(i), l, 1.f, dW, n, s));   // dW += dY Z_i^T
    TIMED(plan, LRAMM_K_SKETCH, s, x_product(plan, ws, *sw.S, 1, W, k, n, d.ldb, sw.xbf, dY, dZ, s));   // dZ = W^T dY
    TIMED(plan, LRAMM_K_ADJOINT, s, qr_adjoint(plan, ws, Zi(i), n, bl_slot(plan, ws, o - 1, 0), nullptr, dZ, dY, s));
    TIMED(plan, LRAMM_K_BWD, s, nt_product(plan, ws, k, n, l, 1.f, Qi(i - 1), l, dY, l, 1.f, dW, n, s));  // dW += Q_{i-1} dY'^T
    TIMED(plan, LRAMM_K_SKETCH, s, x_product(plan, ws, *sw.S, 0, W, k, n, d.ldb, sw.xbf, dY, dQ, s));   // dQ = W dY'
  }
  TIMED(plan, LRAMM_K_ADJOINT, s,
        qr_adjoint(plan, ws, Qi(0), k, bl_slot(plan, ws, 0, 0), d.q == 0 ? bl_slot(plan, ws, 0, 1) : nullptr, dQ, dY, s));
  const float* Om = at<float>(ws, sw.S->omega);
  TIMED(plan, LRAMM_K_BWD, s, nt_product(plan, ws, k, n, l, 1.f, dY, l, Om, l, 1.f, dW, n, s));   // dW += dY_0 Omega^T
  return LRAMM_OK;
}

size_t lramm_qgemm_tc_ws_bytes(int32_t prec, int64_t M, int64_t N, int64_t K) {
  if (M <= 0 || N <= 0 || K <= 0 || (prec != LRAMM_P_INT8 && prec != LRAMM_P_INT4 && prec != LRAMM_P_E4M3))
    return kAlign;
  return kAlign + sizeof(float) * qgemm_tc_part_floats(prec, M, N, K);
}

lramm_status lramm_qgemm_tc(int32_t prec, const void* L, const void* Rt, int64_t M, int64_t N, int64_t K, int64_t ldl,
                            int64_t ldr, int32_t per_row, const float* sL, const float* sR, float alpha, float beta,
                            const float* C, int64_t ldc, float* D, int64_t ldd, void* ws, size_t ws_bytes,
                            void* stream) {
  if (prec != LRAMM_P_INT8 && prec != LRAMM_P_INT4 && prec != LRAMM_P_E4M3) return LRAMM_ERR_INVALID_ARG;
  if (M < 0 || N < 0 || K < 0 || K % 16 || ldl < K || ldr < K || ldd < N) return LRAMM_ERR_INVALID_ARG;
  if (M == 0 || N == 0) return LRAMM_OK;
  if (!L || !Rt || !D || !sL || !sR || (beta != 0.f && (!C || ldc < N))) return LRAMM_ERR_INVALID_ARG;
  if (!ws || (reinterpret_cast<uintptr_t>(ws) % kAlign) || ws_bytes < lramm_qgemm_tc_ws_bytes(prec, M, N, K))
    return LRAMM_ERR_WORKSPACE;
  if (!qgemm_tc_supported(prec, L, Rt, ldl, ldr, M, N, K)) return LRAMM_ERR_UNSUPPORTED;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int* st = static_cast<int*>(ws);
  LRAMM_CUDA_TRY(cudaMemsetAsync(st, 0, sizeof(int) * 4, s));
  float* part = reinterpret_cast<float*>(static_cast<char*>(ws) + kAlign);
  return qgemm_tc(prec, L, Rt, M, N, K, ldl, ldr, per_row, sL, sR, alpha, beta, C, ldc, D, ldd, part,
                  (ws_bytes - kAlign) / sizeof(float), st, s);
}

size_t lramm_tgemm_tc_ws_bytes(int64_t M, int64_t N, int64_t K) {
  if (M <= 0 || N <= 0 || K <= 0) return kAlign;
  return kAlign + sizeof(float) * tgemm_tc_part_floats(M, N, K);
}

lramm_status lramm_tgemm_tc(int64_t M, int64_t N, int64_t K, float alpha, const float* A, int64_t lda, const float* B,
                            int64_t ldb, float beta, float* C, int64_t ldc, void* ws, size_t ws_bytes, void* stream) {
  if (M < 0 || N < 0 || K < 0 || lda < K || ldb < K || ldc < N) return LRAMM_ERR_INVALID_ARG;
  if (M == 0 || N == 0) return LRAMM_OK;
  if (!A || !B || !C) return LRAMM_ERR_INVALID_ARG;
  if (!ws || (reinterpret_cast<uintptr_t>(ws) % kAlign) || ws_bytes < lramm_tgemm_tc_ws_bytes(M, N, K))
    return LRAMM_ERR_WORKSPACE;
  if (K == 0 || !tgemm_tc_supported(A, B, lda, ldb, M, N, K)) return LRAMM_ERR_UNSUPPORTED;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int* st = static_cast<int*>(ws);
  LRAMM_CUDA_TRY(cudaMemsetAsync(st, 0, sizeof(int) * 4, s));
  float* part = reinterpret_cast<float*>(static_cast<char*>(ws) + kAlign);
  return tgemm_tc(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, part, (ws_bytes - kAlign) / sizeof(float), st, s);
}

lramm_status lramm_quantize_mx(const float* X, int64_t rows, int64_t cols, int64_t ldx, int8_t* codes,
                               int64_t ldcodes, int8_t* exps, void* stream) {
  if (rows < 0 || cols < 0 || ldx < cols || ldcodes < cols || ldcodes % 32) return LRAMM_ERR_INVALID_ARG;
  if (rows > 0 && (!X || !codes || !exps)) return LRAMM_ERR_INVALID_ARG;
  return quantize_mx(X, rows, cols, ldx, codes, ldcodes, exps, static_cast<cudaStream_t>(stream));
}

lramm_status lramm_qgemm_mx(const int8_t* L, const int8_t* Le, const int8_t* Rt, const int8_t* Re, int64_t M,
                            int64_t N, int64_t K, int64_t ldl, int64_t ldr, float alpha, float beta, const float* C,
                            int64_t ldc, float* D, int64_t ldd, void* stream) {
  if (M < 0 || N < 0 || K < 0 || K % 32 || ldl < K || ldr < K || ldd < N) return LRAMM_ERR_INVALID_ARG;
  if (M == 0 || N == 0) return LRAMM_OK;
  if (!L || !Le || !Rt || !Re || !D || (beta != 0.f && (!C || ldc < N))) return LRAMM_ERR_INVALID_ARG;
  return qgemm_mx(L, Le, Rt, Re, M, N, K, ldl, ldr, alpha, beta, C, ldc, D, ldd, static_cast<cudaStream_t>(stream));
}

// Direct QM(A B) of Algorithm 2 (the paper's DQ8 / DQ4 comparators).
size_t lramm_dq_ws_bytes(int32_t prec, int64_t m, int64_t n, int64_t k) {
  if (m <= 0 || n <= 0 || k <= 0 || (prec != LRAMM_P_INT8 && prec != LRAMM_P_INT4 && prec != LRAMM_P_E4M3))
    return kAlign;
  const int64_t kp = round_up(k, 32);
  Bump b;
  b.take(kAlign);                                  // status word
  b.take(kAlign);                                  // tensor a_max
  b.take(2 * m * kp);                              // codes of A (widest container)
  b.take(2 * n * kp);                              // codes of B^T
  b.take(sizeof(float) * (m + n));                 // scales
  b.take(sizeof(float) * std::max<size_t>(qgemm_tc_part_floats(prec, m, n, kp), 4));
  return b.off;
}

lramm_status lramm_dq_matmul(int32_t prec, int32_t scale, int64_t m, int64_t n, int64_t k, float alpha,
                             const float* A, int64_t lda, const float* B, int64_t ldb, float beta, const float* C,
                             int64_t ldc, float* D, int64_t ldd, void* ws, size_t ws_bytes, void* stream) {
  if (prec != LRAMM_P_INT8 && prec != LRAMM_P_INT4 && prec != LRAMM_P_E4M3) return LRAMM_ERR_INVALID_ARG;
  if (scale != LRAMM_S_ROWCOL && scale != LRAMM_S_TENSOR) return LRAMM_ERR_INVALID_ARG;
  if (m < 0 || n < 0 || k < 1 || lda < k || ldb < n || ldd < n) return LRAMM_ERR_INVALID_ARG;
  if (m == 0 || n == 0) return LRAMM_OK;
  if (!A || !B || !D || (beta != 0.f && (!C || ldc < n))) return LRAMM_ERR_INVALID_ARG;
  if (!ws || (reinterpret_cast<uintptr_t>(ws) % kAlign) || ws_bytes < lramm_dq_ws_bytes(prec, m, n, k))
    return LRAMM_ERR_WORKSPACE;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int64_t kp = round_up(k, 32);
  const int per = scale == LRAMM_S_ROWCOL;
  Bump b;
  const size_t o_st = b.take(kAlign), o_am = b.take(kAlign), o_ca = b.take(2 * m * kp), o_cb = b.take(2 * n * kp);
  const size_t o_s = b.take(sizeof(float) * (m + n));
  const size_t pf = std::max<size_t>(qgemm_tc_part_floats(prec, m, n, kp), 4);
  const size_t o_p = b.take(sizeof(float) * pf);
  int* st = at<int>(ws, o_st);
  LRAMM_CUDA_TRY(cudaMemsetAsync(st, 0, sizeof(int) * 4, s));
  void* cA = at<void>(ws, o_ca);
  void* cB = at<void>(ws, o_cb);
  float* sA = at<float>(ws, o_s);
  float* sB = sA + m;
  LRAMM_TRY(quantize_rows(A, m, k, lda, prec, per, cA, kp, sA, at<unsigned int>(ws, o_am), s));
  LRAMM_TRY(quantize_cols(B, k, n, ldb, prec, per, cB, kp, sB, at<unsigned int>(ws, o_am), s));
  if (qgemm_tc_supported(prec, cA, cB, kp, kp, m, n, kp))
    return qgemm_tc(prec, cA, cB, m, n, kp, kp, kp, per, sA, sB, alpha, beta, C, ldc, D, ldd, at<float>(ws, o_p), pf,
                    st, s);
  return qgemm(cA, cB, m, n, kp, kp, kp, prec, per, sA, sB, alpha, beta, C, ldc, D, ldd, 0, s);
}

}  // extern "C"
