// capi.cu -- the extern "C" boundary declared in include/he_gb300.h: argument
// checking, context set-up (primes, roots, twiddle tables, constants), buffer
// sizing, the default blocking, launch bookkeeping and event profiling.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/he_gb300.h"
#include "coset.cuh"
#include "kernels.h"
#include "mac_tc.cuh"
#include "mac_tcr.cuh"
#include "multi.h"
#include "ntt.cuh"

using he::u32;
using he::u64;
typedef unsigned __int128 u128;

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

int cuda_fail(cudaError_t e, const char* where) {
  return fail(HE_ECUDA, std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
}

// ---------------------------------------------------------------- host modular arithmetic

u64 mulm(u64 a, u64 b, u64 q) { return (u64)((u128)a * b % q); }

u64 powm(u64 b, u64 e, u64 q) {
  u64 r = 1 % q;
  b %= q;
  for (; e; e >>= 1) {
    if (e & 1) r = mulm(r, b, q);
    b = mulm(b, b, q);
  }
  return r;
}

u64 invm(u64 a, u64 q) { return powm(a, q - 2, q); }  // q prime

bool prime64(u64 n) {
  if (n < 2) return false;
  const u64 small[] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
  for (u64 p : small)
    if (n % p == 0) return n == p;
  u64 d = n - 1;
  int r = 0;
  while (!(d & 1)) d >>= 1, ++r;
  for (u64 a : small) {
    u64 x = powm(a, d, n);
    if (x == 1 || x == n - 1) continue;
    bool comp = true;
    for (int i = 1; i < r && comp; ++i) {
      x = mulm(x, x, n);
      if (x == n - 1) comp = false;
    }
    if (comp) return false;
  }
  return true;
}

// The smallest primitive 2N-th root of unity mod q (all of them are the odd powers of one).
u64 min_root_2n(u64 q, u32 N) {
  u64 base = 0;
  for (u64 g = 2; g < 1000 && !base; ++g) {
    u64 c = powm(g, (q - 1) / (2 * (u64)N), q);
    if (powm(c, N, q) == q - 1) base = c;
  }
  if (!base) return 0;
  u64 best = base, sq = mulm(base, base, q), cur = base;
  for (u32 e = 1; e < N; ++e) {  // odd powers base^(2e+1)
    cur = mulm(cur, sq, q);
    if (cur < best) best = cur;
  }
  return best;
}

u64 shoup(u64 w, u64 q) { return (u64)(((u128)w << 64) / q); }

u32 brev(u32 x, u32 bits) {
  u32 r = 0;
  for (u32 i = 0; i < bits; ++i) r |= ((x >> i) & 1u) << (bits - 1 - i);
  return r;
}

// floor(2^e / q) for 64 < e < 192 with q < 2^63, as a 128-bit value (caller ensures it fits).
u128 pow2_div(u32 e, u64 q) {
  u128 quo = 0, rem = 0;
  for (int bit = (int)e; bit >= 0; --bit) {
    rem = (rem << 1) | (bit == (int)e ? 1 : 0);
    quo <<= 1;
    if (rem >= q) {
      rem -= q;
      quo |= 1;
    }
  }
  return quo;
}

bool pow2(u64 x) { return x && !(x & (x - 1)); }

u32 ceil_div(u32 a, u32 b) { return (a + b - 1) / b; }

}  // namespace

// ---------------------------------------------------------------- context

struct ProfRec {
  int kind;
  cudaEvent_t e0, e1;
};

enum Kind {
  KNttFwd, KNttInv, KPolyMul, KKeygen, KEncrypt, KDecrypt, KPack, KUnpack, KUnmask, KEncode, KMac, KInttMask, KInttC0,
  KExpand, KProbe, KShare, KInvC0, KCheck, KMacTc, KCosetFwd, KCosetInv, KCosetEnc, KCount
};
static const char* kKindNames[KCount] = {"ntt_forward", "ntt_inverse", "poly_mul", "keygen", "encrypt",
                                         "decrypt", "pack", "unpack", "unmask", "encode_weights",
                                         "mac", "intt_mask", "intt_c0_targets", "expand_compact", "probe",
                                         "share_matmul", "intt_c1_c0", "check_residues", "mac_tc",
                                         "coset_forward", "coset_inverse", "coset_encode"};

struct he_ctx {
  int device = 0;
  he::Consts C{};
  u64 psi[he::kMaxPrimes] = {};
  u64* d_tables = nullptr;
  int* d_err = nullptr;  // set by kernels whose bounded waits expired
  uint32_t mac_engine = HE_MAC_AUTO;  // which multiply-accumulate products use (he_set_mac_engine)
  u64* d_bad = nullptr;  // he_ct_import: count and first index of residues out of range
  std::atomic<uint64_t> launches{0};
  bool prof = false;
  std::vector<ProfRec> recs;
  std::vector<cudaEvent_t> pool;
  uint64_t stat_launches[KCount] = {};
  double stat_ms[KCount] = {};
};

namespace {

cudaEvent_t get_event(he_ctx* c) {
  if (!c->pool.empty()) {
    cudaEvent_t e = c->pool.back();
    c->pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Runs one launcher under the context's bookkeeping (launch count, optional events).
template <typename F>
int launch(he_ctx* c, int kind, cudaStream_t st, const char* where, F&& f) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (c->prof) {
    e0 = get_event(c);
    e1 = get_event(c);
    cudaEventRecord(e0, st);
  }
  cudaError_t e = f();
  if (c->prof) {
    cudaEventRecord(e1, st);
    c->recs.push_back({kind, e0, e1});
  }
  c->launches.fetch_add(1, std::memory_order_relaxed);
  if (e != cudaSuccess) return cuda_fail(e, where);
  return HE_OK;
}

int set_device(const he_ctx* c) {
  cudaError_t e = cudaSetDevice(c->device);
  return e == cudaSuccess ? HE_OK : cuda_fail(e, "cudaSetDevice");
}

int check_blk(const he_ctx* c, const he_blocking* b) {
  if (!b) return fail(HE_EINVAL, "blocking is NULL");
  if (!b->m_b || !b->k_b || !b->n_b) return fail(HE_EINVAL, "blocking entries must be >= 1");
  if ((u64)b->m_b * b->k_b * b->n_b > c->C.N) return fail(HE_EINVAL, "blocking needs m_b * k_b * n_b <= N");
  return HE_OK;
}

struct Shape {
  u32 nI, nJ, nLb;
};

Shape shape_of(u32 m, u32 k, u32 n, const he_blocking* b) {
  return {ceil_div(n, b->n_b), ceil_div(k, b->k_b), ceil_div(m, b->m_b)};
}

he::Blk to_blk(const he_blocking* b) { return {b->m_b, b->k_b, b->n_b}; }

// Whether a product with nJ k-blocks uses the tensor-core multiply-accumulate (and its
// stage-tiled operand layout) on this context: needs N >= 512; HE_MAC_AUTO takes it from
// kTcMinKBlocks k-blocks on, where the exact limb split amortises its digit split and
// epilogue; HE_MAC_TENSOR for every product; HE_MAC_INTEGER never.
constexpr u32 kTcMinKBlocks = 32;

// Whether a product under blocking b runs through the ring's cosets (coset.cuh): weight
// blocks of 2D residues instead of N, D = max(8, next power of two of n_b k_b) <= N/2, on the
// tensor-core multiply-accumulate.  HE_MAC_AUTO and HE_MAC_COSET take it wherever it applies
// (N >= 512).
bool use_coset(const he_ctx* c, const he_blocking* b) {
  if (c->C.logN < 9 || (c->mac_engine != HE_MAC_AUTO && c->mac_engine != HE_MAC_COSET)) return false;
  return he::coset_logD(b->n_b * b->k_b) < c->C.logN;
}
// Coset products of at most 64 k-blocks run the row-major tensor-core MAC (mac_tcr.cuh):
// inputs on the MMA's M, every weight tile streamed past them.
bool use_tcr(const he_ctx* c, const he_blocking* b, u32 nJ) {
  return use_coset(c, b) && nJ <= he::kTcrMaxStages * he::kTcJB;
}
bool use_tc(const he_ctx* c, const he_blocking* b, u32 nJ) {
  if (c->C.logN < 9 || c->mac_engine == HE_MAC_INTEGER) return false;
  if (use_coset(c, b)) return true;
  return c->mac_engine == HE_MAC_TENSOR || c->mac_engine == HE_MAC_COSET || nJ >= kTcMinKBlocks;
}

// Geometry of a coset product: 2D slots per prime, rows (2 Lb + c) G + g.
struct CosetGeom {
  u32 logD, S, R;
  u64 ctn_words, acc_words;
};
CosetGeom coset_geom(const he_ctx* c, const he_blocking* b, u32 nI, u32 nJ, u32 nLb) {
  CosetGeom g;
  g.logD = he::coset_logD(b->n_b * b->k_b);
  g.S = 2u << g.logD;
  g.R = (2 * nLb) << (c->C.logN - g.logD);
  g.ctn_words = he::tc_words(g.R, nJ, c->C.L, g.S);
  g.acc_words = (u64)nLb * nI * 2 * c->C.L * 2 * c->C.N;
  return g;
}
u64 up256(u64 b) { return (b + 255) & ~(u64)255; }

// Words of the NTT of a product's inputs (2 nLb rows) and of its encoded weights (nI rows) in
// the layout of its multiply-accumulate: the tensor-core one pads k-blocks to stages of 16 and
// stores the weights as bf16 digit tiles; coset products have 2D slots per prime (and G times
// the input rows).
u64 operand_words(const he_ctx* c, const he_blocking* b, u32 rows, u32 nJ) {
  if (use_coset(c, b)) return coset_geom(c, b, 0, nJ, rows / 2).ctn_words;
  return use_tc(c, b, nJ) ? he::tc_words(rows, nJ, c->C.L, c->C.N) : (u64)rows * nJ * c->C.L * c->C.N;
}
u64 weight_words(const he_ctx* c, const he_blocking* b, u32 nI, u32 nJ) {
  if (use_coset(c, b)) {
    const u32 S = 2u << he::coset_logD(b->n_b * b->k_b);
    return use_tcr(c, b, nJ) ? he::tcr_weight_words(nI, nJ, c->C.L, S) : he::tc_weight_words(nI, nJ, c->C.L, S);
  }
  return use_tc(c, b, nJ) ? he::tc_weight_words(nI, nJ, c->C.L, c->C.N) : (u64)nI * nJ * c->C.L * c->C.N;
}

}  // namespace

extern "C" {

const char* he_last_error(void) { return g_last_error.c_str(); }

int he_params_init(he_ctx** out, uint32_t N, uint32_t L, const uint64_t* q, uint32_t log2_t, int device) {
  if (!out) return fail(HE_EINVAL, "ctx out-pointer is NULL");
  *out = nullptr;
  if (!pow2(N) || N < 32 || N > 8192) return fail(HE_EINVAL, "N must be a power of two in [32, 8192]");
  if (L < 1 || L > (u32)he::kMaxPrimes || (u64)L * N > 3ull * 8192)
    return fail(HE_EINVAL, "L must be in [1, 3] with L * N <= 3 * 8192");
  if (!q) return fail(HE_EINVAL, "prime array is NULL");
  if (log2_t < 2 || log2_t > 48) return fail(HE_EINVAL, "log2_t must be in [2, 48]");
  for (u32 l = 0; l < L; ++l) {
    if (q[l] >= (1ull << 50) || q[l] <= (1ull << log2_t)) return fail(HE_EINVAL, "need 2^log2_t < q_l < 2^50");
    if ((q[l] - 1) % (2ull * N)) return fail(HE_EINVAL, "q_l must be 1 mod 2N");
    if ((q[l] & 0xffffffffull) != 1) return fail(HE_EINVAL, "q_l must be 1 mod 2^32 (q_l = c 2^32 + 1)");
    if (!prime64(q[l])) return fail(HE_EINVAL, "q_l must be prime");
    for (u32 j = 0; j < l; ++j)
      if (q[j] == q[l]) return fail(HE_EINVAL, "primes must be distinct");
  }
  if (device < 0) return fail(HE_EINVAL, "device must be >= 0");

  he_ctx* c = new he_ctx();
  c->device = device;
  he::Consts& C = c->C;
  C.N = N;
  C.logN = 0;
  while ((1u << C.logN) < N) ++C.logN;
  C.L = L;
  C.log2t = log2_t;
  C.logR = he::kNttLogRDefault;
  C.tmask = (1ull << log2_t) - 1;
  u64 qmt = 1;
  for (u32 l = 0; l < L; ++l) qmt = (u64)(((u128)qmt * (q[l] & C.tmask)) & C.tmask);
  C.q_mod_t = qmt;

  constexpr u32 kTableWords = 6;  // per prime: 4N twiddle words, then 2N words of coset fold factors
  std::vector<u64> host((size_t)kTableWords * L * N);
  for (u32 l = 0; l < L; ++l) {
    const u64 ql = q[l];
    he::PrimeConsts& P = C.p[l];
    u64 psi = min_root_2n(ql, N);
    if (!psi) {
      delete c;
      return fail(HE_EINVAL, "no primitive 2N-th root found");
    }
    c->psi[l] = psi;
    u64 ipsi = invm(psi, ql);
    u64* tw = host.data() + (size_t)kTableWords * l * N;
    for (u32 kk = 0; kk < N; ++kk) {
      u32 e = brev(kk, C.logN);
      tw[kk] = powm(psi, e, ql);
      tw[N + kk] = shoup(tw[kk], ql);
      tw[2 * N + kk] = powm(ipsi, e, ql);
      tw[3 * N + kk] = shoup(tw[2 * N + kk], ql);
    }
    // coset fold factors (1 +- psi^{brev(k)} psi^{-N/2}) / (2N), k < N/2 (coset.cuh)
    const u64 inv2n = invm((2ull * N) % ql, ql), w_half = tw[2 * N + 1];
    for (u32 kk = 0; kk < N / 2; ++kk) {
      const u64 zw = mulm(tw[kk], w_half, ql);
      u64* f = tw + 4 * N + 4 * kk;
      f[0] = mulm((1 + zw) % ql, inv2n, ql);
      f[1] = shoup(f[0], ql);
      f[2] = mulm((1 + ql - zw) % ql, inv2n, ql);
      f[3] = shoup(f[2], ql);
    }
    P.q = ql;
    P.two_q = 2 * ql;
    P.mu = shoup(1, ql);
    P.ninv = invm(N % ql, ql);
    P.ninv_sh = shoup(P.ninv, ql);
    P.tinv = invm((1ull << log2_t) % ql, ql);
    P.tinv_sh = shoup(P.tinv, ql);
    P.r25 = (1ull << 25) % ql;
    P.r25_sh = shoup(P.r25, ql);
    P.r32 = 1ull << 32;
    P.r32_sh = shoup(P.r32, ql);
    P.r50 = (1ull << 50) % ql;
    P.r50_sh = shoup(P.r50, ql);
    P.r64 = (u64)(((u128)1 << 64) % ql);
    P.r64_sh = shoup(P.r64, ql);
    u64 pw = 1, pw_sum = 0;
    for (u32 d = 0; d < 13; ++d) {  // 256^d mod q < 2^50: high halves below 2^18
      P.pw256_lo[d] = (uint32_t)pw;
      P.pw256_hi[d] = (uint32_t)(pw >> 32);
      pw_sum = (pw_sum + pw) % ql;
      pw = mulm(pw, 256, ql);
    }
    P.pw256_bias = mulm((1ull << 24) % ql, pw_sum, ql);
    u64 Ml = 1;
    for (u32 j = 0; j < L; ++j)
      if (j != l) Ml = mulm(Ml, q[j] % ql, ql);
    P.crt = invm(Ml, ql);
    P.crt_sh = shoup(P.crt, ql);
    u128 theta = pow2_div(128 + log2_t, ql);
    P.theta_hi = (u64)(theta >> 64);
    P.theta_lo = (u64)theta;
  }

  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) {
    delete c;
    return cuda_fail(e, "cudaSetDevice");
  }
  e = cudaMalloc(&c->d_tables, host.size() * sizeof(u64));
  if (e == cudaSuccess) e = cudaMalloc(&c->d_err, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&c->d_bad, 2 * sizeof(u64));
  if (e != cudaSuccess) {
    if (c->d_tables) cudaFree(c->d_tables);
    if (c->d_err) cudaFree(c->d_err);
    delete c;
    return fail(HE_ENOMEM, "cudaMalloc of context tables failed");
  }
  e = cudaMemset(c->d_err, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaMemcpy(c->d_tables, host.data(), host.size() * sizeof(u64), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = he::configure_kernels(C);
  if (e == cudaSuccess) e = he::configure_multi_kernels();
  if (e != cudaSuccess) {
    cudaFree(c->d_tables);
    cudaFree(c->d_err);
    cudaFree(c->d_bad);
    delete c;
    return cuda_fail(e, "table upload / kernel configuration");
  }
  for (u32 l = 0; l < L; ++l) {
    u64* tw = c->d_tables + (size_t)kTableWords * l * N;
    C.p[l].psi = tw;
    C.p[l].psi_sh = tw + N;
    C.p[l].ipsi = tw + 2 * N;
    C.p[l].ipsi_sh = tw + 3 * N;
    C.p[l].fold = tw + 4 * N;
  }
  *out = c;
  return HE_OK;
}

int he_ctx_free(he_ctx* c) {
  if (!c) return HE_OK;
  cudaSetDevice(c->device);
  for (auto& r : c->recs) {
    cudaEventDestroy(r.e0);
    cudaEventDestroy(r.e1);
  }
  for (auto e : c->pool) cudaEventDestroy(e);
  if (c->d_tables) cudaFree(c->d_tables);
  if (c->d_err) cudaFree(c->d_err);
  if (c->d_bad) cudaFree(c->d_bad);
  delete c;
  return HE_OK;
}

int he_get_params(const he_ctx* c, uint32_t* N, uint32_t* L, uint32_t* log2_t, uint64_t* q, uint64_t* psi) {
  if (!c) return fail(HE_EINVAL, "ctx is NULL");
  if (N) *N = c->C.N;
  if (L) *L = c->C.L;
  if (log2_t) *log2_t = c->C.log2t;
  for (u32 l = 0; l < c->C.L; ++l) {
    if (q) q[l] = c->C.p[l].q;
    if (psi) psi[l] = c->psi[l];
  }
  return HE_OK;
}

int he_sizes(const he_ctx* c, uint32_t m, uint32_t k, uint32_t n, const he_blocking* blk, he_size_info* out) {
  if (!c || !out) return fail(HE_EINVAL, "NULL argument");
  int r = check_blk(c, blk);
  if (r) return r;
  Shape s = shape_of(m, k, n, blk);
  const u64 N = c->C.N, L = c->C.L;
  out->nI = s.nI;
  out->nJ = s.nJ;
  out->nLb = s.nLb;
  out->in_cts = (u64)s.nLb * s.nJ;
  out->out_cts = (u64)s.nLb * s.nI;
  out->pts = (u64)s.nI * s.nJ;
  out->in_words = out->in_cts * 2 * L * N;
  out->out_words = out->out_cts * 2 * L * N;
  out->pt_words = weight_words(c, blk, s.nI, s.nJ);
  out->packed_words = out->in_cts * N;
  const u64 Nc = pow2(blk->k_b) ? N / blk->k_b : 0;
  out->out_words_compact = Nc ? out->out_cts * L * (Nc + N) : 0;
  if (use_coset(c, blk)) {  // the inputs' coset transforms, then the sums of both components
    const CosetGeom g = coset_geom(c, blk, s.nI, s.nJ, s.nLb);
    out->workspace_bytes = out->workspace_bytes_compact = up256(g.ctn_words * 8) + up256(g.acc_words * 8);
    return HE_OK;
  }
  const u64 ntt_words = operand_words(c, blk, 2 * s.nLb, s.nJ);  // NTT of the input ciphertexts (MAC layout)
  out->workspace_bytes = ntt_words * sizeof(u64);
  out->workspace_bytes_compact = (ntt_words + out->out_cts * L * N) * sizeof(u64);
  return HE_OK;
}

namespace {

struct Candidate {
  he_blocking b;
  double cost;  // model seconds
};

// Every power-of-two blocking of an (m x k) . (k x n) product with m_b k_b n_b <= N and
// no block larger than the next power of two of its dimension, sorted by a cost model of
// one product on GB300 (seconds; constants measured with bench.py):
//   transforms: 45 ns per length-4096 residue polynomial (scaled by N log N), counting the
//     NTT of every input polynomial, the inverse NTT of every output polynomial and, when
//     the weights are encoded per call, the NTT of every weight polynomial;
//   multiply-accumulate on the integer pipe: 0.8 ps per slot product, divided by the fill of
//     the kernel's 8-row x 8-column output tiles;
//   multiply-accumulate on the tensor cores (where the engine puts the product there): 0.07
//     ps per slot product divided by the fill of its 128-weight-row x 16-row work units,
//     plus the weights' digit form (14 instead of 8 bytes per residue; when encoded per
//     call also cleared and written in that form);
//   memory: algorithmic bytes at 6.75 TB/s;
//   coset products (where the engine puts the product there, coset.cuh): 2N slot products per
//     input block, weight block and component; transforms of the inputs and the outputs
//     scaled by their stages, (log2 G + 2 log2 D) / log2 N, with 2N words each in the
//     transform domain; weights of 2D slots in digit form; the multiply-accumulate's
//     epilogue (3 ps per output word and accumulation round of 128 k-blocks) overlapping its
//     MMAs.
// Ties go to the larger m_b, then the larger k_b.
std::vector<Candidate> blocking_candidates(u32 Nw, u32 Lw, u32 m, u32 k, u32 n, u32 weights_per_call,
                                           u32 engine = HE_MAC_AUTO) {
  const double N = Nw, L = Lw;
  const double t_poly = 45e-9 * (N * std::log2(N)) / (4096.0 * 12.0);
  const double t_slot = 0.8e-12, t_slot_tc = 0.07e-12, hbm = 6.75e12;
  auto cap = [&](u32 d) {
    u64 p = 1;
    while (p < d && p < Nw) p <<= 1;
    return p;
  };
  const u64 cm = cap(m ? m : 1), ck = cap(k ? k : 1), cn = cap(n ? n : 1);
  std::vector<Candidate> out;
  for (u64 mb = 1; mb <= cm; mb <<= 1)
    for (u64 kb = 1; kb <= ck && mb * kb <= Nw; kb <<= 1)
      for (u64 nb = 1; nb <= cn && mb * kb * nb <= Nw; nb <<= 1) {
        const double nI = (double)((n + nb - 1) / nb), nJ = (double)((k + kb - 1) / kb),
                     nLb = (double)((m + mb - 1) / mb);
        if (nJ > 4096) continue;
        const double pts = nI * nJ, in = nLb * nJ, outc = nLb * nI;
        const double polys = 2 * L * in + 2 * L * outc + (weights_per_call ? L * pts : 0);
        const double rows = 2 * nLb, slots = nI * nJ * nLb * 2 * L * N;
        const u32 logD = he::coset_logD((u32)(kb * nb));
        if (Nw >= 512 && (engine == HE_MAC_AUTO || engine == HE_MAC_COSET) && (1u << logD) <= Nw / 2) {
          const double D = (double)(1u << logD), G = N / D, S = 2 * D, R = rows * G;
          const double nS = std::ceil(nJ / 16.0);
          const double fill = (R / (16 * std::ceil(R / 16))) * (nI / (128 * std::ceil(nI / 128)));
          const double mma = 2 * slots * (16 * nS / nJ) * t_slot_tc / fill;
          const double epi = 3e-12 * R * nI * S * L * std::ceil(nS / 8);
          const double xf = t_poly * (std::log2(G) + 2 * std::log2(D)) / std::log2(N) * 1.5;
          const double cbytes = 8 * N * L * (10 * in + 10 * outc) + 14 * S * L * pts * (weights_per_call ? 2 : 1) +
                                (weights_per_call ? 8.0 * k * n : 0);
          out.push_back({{(u32)mb, (u32)kb, (u32)nb},
                         (2 * L * in + 2 * L * outc + (weights_per_call ? L * pts * S / N : 0)) * xf +
                             std::max(mma, epi) + cbytes / hbm});
          continue;
        }
        const bool tc = Nw >= 512 && engine != HE_MAC_INTEGER &&
                        (engine == HE_MAC_TENSOR || engine == HE_MAC_COSET || nJ >= 32);
        double bytes = 8 * N * L * (pts * (weights_per_call ? 3 : 1) + 6 * in + 4 * outc), mac;
        if (tc) {
          const double fill = (rows / (16 * std::ceil(rows / 16))) * (nI / (128 * std::ceil(nI / 128)));
          mac = slots * t_slot_tc / fill;
          bytes += N * L * pts * (weights_per_call ? 34 : 6);
        } else {
          const double fill = (rows / (8 * std::ceil(rows / 8))) * (nI / (8 * std::ceil(nI / 8)));
          mac = slots * t_slot / fill;
        }
        out.push_back({{(u32)mb, (u32)kb, (u32)nb}, polys * t_poly + mac + bytes / hbm});
      }
  std::stable_sort(out.begin(), out.end(), [](const Candidate& a, const Candidate& b) {
    if (a.cost < b.cost * (1 - 1e-9)) return true;
    if (b.cost < a.cost * (1 - 1e-9)) return false;
    return a.b.m_b != b.b.m_b ? a.b.m_b > b.b.m_b : a.b.k_b > b.b.k_b;
  });
  return out;
}

}  // namespace

int he_choose_blocking(uint32_t Nw, uint32_t Lw, uint32_t m, uint32_t k, uint32_t n, uint32_t weights_per_call,
                       he_blocking* out) {
  if (!out) return fail(HE_EINVAL, "NULL argument");
  if (!pow2(Nw) || Lw < 1) return fail(HE_EINVAL, "N must be a power of two and L >= 1");
  const std::vector<Candidate> c = blocking_candidates(Nw, Lw, m, k, n, weights_per_call);
  *out = c.empty() ? he_blocking{1, 1, 1} : c.front().b;
  return HE_OK;
}

int he_default_blocking(const he_ctx* c, uint32_t m, uint32_t k, uint32_t n, uint32_t weights_per_call,
                        he_blocking* out) {
  if (!c || !out) return fail(HE_EINVAL, "NULL argument");
  if (!pow2(c->C.N)) return fail(HE_EINVAL, "N must be a power of two");
  const std::vector<Candidate> cand = blocking_candidates(c->C.N, c->C.L, m, k, n, weights_per_call, c->mac_engine);
  if (cand.empty()) return fail(HE_EINVAL, "no blocking fits");
  *out = cand.front().b;
  return HE_OK;
}

int he_keygen(he_ctx* c, uint64_t seed, uint64_t* sk, void* stream) {
  if (!c || !sk) return fail(HE_EINVAL, "NULL argument");
  if (int r = set_device(c)) return r;
  return launch(c, KKeygen, (cudaStream_t)stream, "keygen",
                [&] { return he::launch_keygen(c->C, seed, sk, (cudaStream_t)stream); });
}

int he_encrypt(he_ctx* c, const uint64_t* sk, const uint64_t* plain, uint32_t cnt, uint64_t seed, uint64_t* ct,
               void* stream) {
  if (!c) return fail(HE_EINVAL, "ctx is NULL");
  if (!cnt) return HE_OK;
  if (!sk || !plain || !ct) return fail(HE_EINVAL, "NULL buffer");
  if (int r = set_device(c)) return r;
  return launch(c, KEncrypt, (cudaStream_t)stream, "encrypt",
                [&] { return he::launch_encrypt(c->C, sk, plain, cnt, seed, ct, (cudaStream_t)stream); });
}

int he_decrypt(he_ctx* c, const uint64_t* sk, const uint64_t* ct, uint32_t cnt, uint64_t* plain,
               int32_t* noise_budget, int32_t* min_budget_host, void* stream) {
  if (!c) return fail(HE_EINVAL, "ctx is NULL");
  if (min_budget_host) *min_budget_host = 63;
  if (!cnt) return HE_OK;
  if (!sk || !ct || !plain) return fail(HE_EINVAL, "NULL buffer");
  if (min_budget_host && !noise_budget) return fail(HE_EINVAL, "min_budget_host needs the noise_budget buffer");
  if (int r = set_device(c)) return r;
  cudaStream_t st = (cudaStream_t)stream;
  int r = launch(c, KDecrypt, st, "decrypt",
                 [&] { return he::launch_decrypt(c->C, sk, ct, cnt, plain, (int*)noise_budget, st); });
  if (r || !min_budget_host) return r;
  std::vector<int32_t> b(cnt);
  cudaError_t e = cudaMemcpyAsync(b.data(), noise_budget, cnt * sizeof(int32_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "decrypt budget readback");
  int32_t mn = 63;
  for (auto v : b) mn = v < mn ? v : mn;
  *min_budget_host = mn;
  return mn <= 0 ? fail(HE_ENOISE, "noise budget exhausted") : HE_OK;
}

int he_pack_input(he_ctx* c, const uint64_t* X, uint32_t m, uint32_t k, const he_blocking* blk, uint64_t* polys,
                  void* stream) {
  if (!c) return fail(HE_EINVAL, "ctx is NULL");
  if (int r = check_blk(c, blk)) return r;
  if (!m || !k) return HE_OK;
  if (!X || !polys) return fail(HE_EINVAL, "NULL buffer");
  if (int r = set_device(c)) return r;
  Shape s = shape_of(m, k, 1, blk);
  return launch(c, KPack, (cudaStream_t)stream, "pack", [&] {
    return he::launch_pack(c->C, X, m, k, to_blk(blk), s.nJ, s.nLb, polys, (cudaStream_t)stream);
  });
}

int he_unpack_output(he_ctx* c, const uint64_t* dec, uint32_t m, uint32_t n, const he_blocking* blk,
                     uint64_t* client_share, void* stream) {
  if (!c) return fail(HE_EINVAL, "ctx is NULL");
  if (int r = check_blk(c, blk)) return r;
  if (!m || !n) return HE_OK;
  if (!dec || !client_share) return fail(HE_EINVAL, "NULL buffer");
  if (int r = set_device(c)) return r;
  Shape s = shape_of(m, 1, n, blk);
  return launch(c, KUnpack, (cudaStream_t)stream, "unpack", [&] {
    return he::launch_unpack(c->C, dec, m, n, to_blk(blk), s.nI, client_share, (cudaStream_t)stream);
  });
}

int he_unmask(he_ctx* c, uint64_t mask_seed, uint32_t m, uint32_t n, const he_blocking* blk, uint64_t* server_share,
              void* stream) {
  if (!c) return fail(HE_EINVAL, "ctx is NULL");
  if (int r = check_blk(c, blk)) return r;
  if (!m || !n) return HE_OK;
  if (!server_share) return fail(HE_EINVAL, "NULL buffer");
  if (int r = set_device(c)) return r;
  Shape s = shape_of(m, 1, n, blk);
  return launch(c, KUnmask, (cudaStream_t)stream, "unmask", [&] {
    return he::launch_unmask(c->C, mask_seed, m, n, to_blk(blk), s.nI, server_share, (cudaStream_t)stream);
  });
}

int he_unmask_acc(he_ctx* c, uint64_t mask_seed, uint32_t m, uint32_t n, const he_blocking* blk, uint32_t flags,
                  uint64_t* out, void* stream) {
  if (!c) return fail(HE_EINVAL, "ctx is NULL");
  if (int r = check_blk(c, blk)) return r;
  if (flags & ~(HE_UNMASK_ACCUMULATE | HE_UNMASK_TRANSPOSE)) return fail(HE_EINVAL, "unknown flags");
  if (!m || !n) return HE_OK;
  if (!out) return fail(HE_EINVAL, "NULL buffer");
  if (int r = set_device(c)) return r;
  Shape s = shape_of(m, 1, n, blk);
  return launch(c, KUnmask, (cudaStream_t)stream, "unmask_acc", [&] {
    return he::launch_unmask_acc(c->C, mask_seed, m, n, to_blk(blk), s.nI, (flags & HE_UNMASK_ACCUMULATE) != 0,
                                 (flags & HE_UNMASK_TRANSPOSE) != 0, out, (cudaStream_t)stream);
  });
}

int he_share_matmul_batch(he_ctx* c, const uint64_t* X, const uint64_t* W, const uint64_t* bias, const uint64_t* acc,
                          uint32_t m, uint32_t k, uint32_t n, uint32_t batch, uint64_t* out, void* stream) {
  if (!c) return fail(HE_EINVAL, "ctx is NULL");
  if (!m || !n || !batch) return HE_OK;
  if (batch > 65535) return fail(HE_EINVAL, "batch must be <= 65535");
  if (!out || (k && (!X || !W))) return fail(HE_EINVAL, "NULL buffer");
  if (int r = set_device(c)) return r;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
  const u32 splits = k ? he::share_matmul_splits(m, k, n, batch, sms > 0 ? sms : 1) : 1;
  int r = launch(c, KShare, (cudaStream_t)stream, "share_matmul", [&] {
    return he::launch_share_matmul(c->C, X, W, bias, acc, m, k, n, batch, splits, out, (cudaStream_t)stream);
  });
  if (r == HE_OK && splits > 1) c->launches.fetch_add(2, std::memory_order_relaxed);  // set-up + finishing pass
  return r;
}

int he_share_matmul(he_ctx* c, const uint64_t* X, const uint64_t* W, const uint64_t* bias, const uint64_t* acc,
                    uint32_t m, uint32_t k, uint32_t n, uint64_t* out, void* stream) {
  return he_share_matmul_batch(c, X, W, bias, acc, m, k, n, 1, out, stream);
}

int he_encode_weights_batch(he_ctx* c, const uint64_t* W, uint32_t k, uint32_t n, const he_blocking* blk,
                            uint32_t batch, uint64_t* pt, void* stream) {
  if (!c) return fail(HE_EINVAL, "ctx is NULL");
  if (int r = check_blk(c, blk)) return r;
  if (!k || !n || !batch) return HE_OK;
  if (!W || !pt) return fail(HE_EINVAL, "NULL buffer");
  if (int r = set_device(c)) return r;
  Shape s = shape_of(1, k, n, blk);
  if (use_coset(c, blk))
    return launch(c, KCosetEnc, (cudaStream_t)stream, "encode_weights (cosets)", [&] {
      return he::launch_coset_encode_weights(c->C, W, k, n, to_blk(blk), s.nI, s.nJ, batch, use_tcr(c, blk, s.nJ), pt,
                                             (cudaStream_t)stream);
    });
  return launch(c, KEncode, (cudaStream_t)stream, "encode_weights", [&] {
    return he::launch_encode_weights(c->C, W, k, n, to_blk(blk), s.nI, s.nJ, batch, use_tc(c, blk, s.nJ), pt,
                                     (cudaStream_t)stream);
  });
}

int he_encode_weights(he_ctx* c, const uint64_t* W, uint32_t k, uint32_t n, const he_blocking* blk, uint64_t* pt,
                      void* stream) {
  return he_encode_weights_batch(c, W, k, n, blk, 1, pt, stream);
}

static u32 log2u(u32 x) {
  u32 r = 0;
  while ((1u << r) < x) ++r;
  return r;
}

namespace {

// A coset product's entry in a multi-product table (coset.cuh); the begins are the running
// block counts of the three coset grids, advanced past this item.
void coset_item(const he_ctx* c, he::MultiItem& it, const he_blocking* blk, Shape s, bool compact, u64* ws,
                u64* cfwd, u64* tc, u64* tcr, u64* cinv) {
  const CosetGeom g = coset_geom(c, blk, s.nI, s.nJ, s.nLb);
  const u64 L = c->C.L;
  it.nI = s.nI;
  it.nJ = s.nJ;
  it.nLb = s.nLb;
  it.compact = compact;
  it.logkb = compact ? log2u(blk->k_b) : 0;
  it.tc = 1;
  it.coset = 1;
  it.logD = g.logD;
  it.ctN = ws;
  it.acc = ws ? (u64*)((char*)ws + up256(g.ctn_words * 8)) : nullptr;
  it.cfwd_begin = *cfwd;
  it.tc_begin = *tc;
  it.tcr_begin = *tcr;
  it.cinv_begin = *cinv;
  it.tcr = use_tcr(c, blk, s.nJ);
  *cfwd += (u64)s.nLb * s.nJ * 2 * L;
  if (it.tcr) *tcr += he::tcr_units(g.S, (u32)L, g.R);
  else *tc += he::tc_units(g.S, (u32)L, s.nI, g.R);
  *cinv += (u64)s.nLb * s.nI * 2 * L;
}

int launch_coset_grids(he_ctx* c, const he::MultiTable& T, u64 cfwd, u64 tc, u64 tcr, u64 cinv, bool compact,
                       cudaStream_t st) {
  int r = HE_OK;
  if (cfwd)
    r = launch(c, KCosetFwd, st, "coset forward transforms",
               [&] { return he::launch_coset_fwd_multi(c->C, T, cfwd, st); });
  if (!r && tc)
    r = launch(c, KMacTc, st, "tensor-core multiply-accumulate (cosets)",
               [&] { return he::launch_mac_tc_multi(c->C, T, tc, c->d_err, st); });
  if (!r && tcr)
    r = launch(c, KMacTc, st, "row-major tensor-core multiply-accumulate (cosets)",
               [&] { return he::launch_mac_tcr_multi(c->C, T, tcr, c->d_err, st); });
  if (!r && cinv)
    r = launch(c, KCosetInv, st, compact ? "coset inverse transforms + mask (compact)" : "coset inverse transforms + mask",
               [&] { return he::launch_coset_inv_multi(c->C, T, cinv, st); });
  return r;
}

// he_matmul / he_matmul_batch of a coset product: the batch in tables of up to 64 items;
// item b reads its inputs and weights, writes its outputs and uses its workspace at b times
// the per-item sizes, and masks with mask_seed + b.
int coset_matmul(he_ctx* c, const uint64_t* ct_in, const uint64_t* pt, uint32_t m, uint32_t k, uint32_t n,
                 const he_blocking* blk, uint32_t batch, uint64_t mask_seed, uint32_t flags, uint64_t* ct_out,
                 void* ws, cudaStream_t st) {
  he_size_info si;
  he_sizes(c, m, k, n, blk, &si);
  const bool compact = flags & HE_DROP_C0;
  const Shape s = shape_of(m, k, n, blk);
  const u64 out_w = compact ? si.out_words_compact : si.out_words;
  static thread_local he::MultiTable T;
  for (u32 b0 = 0; b0 < batch; b0 += he::kMaxMulti) {
    const u32 cnt = std::min<u32>(he::kMaxMulti, batch - b0);
    memset(&T, 0, sizeof(T));
    T.count = cnt;
    u64 cfwd = 0, tc = 0, tcr = 0, cinv = 0;
    for (u32 i = 0; i < cnt; ++i) {
      const u64 b = b0 + i;
      he::MultiItem& it = T.it[i];
      it.ct_in = ct_in + b * si.in_words;
      it.pt = pt + b * si.pt_words;
      it.out = ct_out + b * out_w;
      it.mask_seed = mask_seed + b;
      coset_item(c, it, blk, s, compact, (u64*)((char*)ws + b * si.workspace_bytes), &cfwd, &tc, &tcr, &cinv);
    }
    if (int r = launch_coset_grids(c, T, cfwd, tc, tcr, cinv, compact, st)) return r;
  }
  return HE_OK;
}

}  // namespace

static int matmul_device(he_ctx* c, const uint64_t* ct_in, const uint64_t* pt, uint32_t m, uint32_t k, uint32_t n,
                         const he_blocking* blk, uint32_t batch, uint64_t mask_seed, uint32_t flags, uint64_t* ct_out,
                         void* ws, cudaStream_t st) {
  if (use_coset(c, blk)) return coset_matmul(c, ct_in, pt, m, k, n, blk, batch, mask_seed, flags, ct_out, ws, st);
  Shape s = shape_of(m, k, n, blk);
  const u64 N = c->C.N, L = c->C.L;
  const u64 out_cts = (u64)s.nLb * s.nI;
  u64* ctN = (u64*)ws;
  const bool tc = use_tc(c, blk, s.nJ);
  auto mac = [&](u64* o0, u64 st0, u64* o1, u64 st1) {
    return tc ? he::launch_mac_tc(c->C, ctN, pt, o0, st0, o1, st1, s.nI, s.nJ, s.nLb, batch, c->d_err, st)
              : he::launch_mac(c->C, ctN, pt, o0, st0, o1, st1, s.nI, s.nJ, s.nLb, batch, c->d_err, st);
  };
  int r = launch(c, KNttFwd, st, "matmul: forward NTT",
                 [&] { return he::launch_ntt_forward_mm(c->C, ct_in, ctN, s.nJ, s.nLb, batch, tc, st); });
  if (r) return r;
  if (!(flags & HE_DROP_C0)) {
    r = launch(c, tc ? KMacTc : KMac, st, "matmul: multiply-accumulate",
               [&] { return mac(ct_out, 2 * L * N, ct_out + L * N, 2 * L * N); });
    if (r) return r;
    return launch(c, KInttMask, st, "matmul: inverse NTT + mask",
                  [&] { return he::launch_intt_mask(c->C, ct_out, out_cts, batch, mask_seed, st); });
  }
  // compact output: per ciphertext [c0 at the decoded coefficients: L x N/k_b][c1: L x N]
  const u32 logkb = log2u(blk->k_b);
  const u64 Nc = N >> logkb, ct_stride = L * (Nc + N);
  u64* c0_ntt = ctN + (u64)batch * operand_words(c, blk, 2 * s.nLb, s.nJ);  // after the inputs' NTT
  r = launch(c, tc ? KMacTc : KMac, st, "matmul: multiply-accumulate",
             [&] { return mac(c0_ntt, L * N, ct_out + L * Nc, ct_stride); });
  if (r) return r;
  r = launch(c, KInttMask, st, "matmul: inverse NTT of c1",
             [&] { return he::launch_intt_c1(c->C, ct_out + L * Nc, ct_stride, out_cts * batch, st); });
  if (r) return r;
  return launch(c, KInttC0, st, "matmul: pruned inverse NTT + mask of c0", [&] {
    return he::launch_intt_c0_targets(c->C, c0_ntt, ct_out, ct_stride, out_cts, batch, logkb, mask_seed, st);
  });
}

static int matmul_checks(he_ctx* c, uint32_t m, uint32_t k, uint32_t n, const he_blocking* blk, uint32_t flags,
                         he_size_info* si) {
  if (!c) return fail(HE_EINVAL, "ctx is NULL");
  if (int r = check_blk(c, blk)) return r;
  if (flags & ~(uint32_t)(HE_DROP_C0 | HE_ASYNC)) return fail(HE_EINVAL, "unknown flags");
  if ((flags & HE_DROP_C0) && !pow2(blk->k_b)) return fail(HE_EINVAL, "HE_DROP_C0 needs a power-of-two k_b");
  he_sizes(c, m, k, n, blk, si);
  if (si->nJ > 4096) return fail(HE_EINVAL, "at most 4096 k-blocks (k / k_b) per product");
  return HE_OK;
}

int he_matmul(he_ctx* c, const uint64_t* ct_in, const uint64_t* pt, uint32_t m, uint32_t k, uint32_t n,
              const he_blocking* blk, uint64_t mask_seed, uint32_t flags, uint64_t* ct_out, void* workspace,
              size_t workspace_bytes, void* stream) {
  he_size_info si;
  if (flags & HE_ASYNC) return fail(HE_EINVAL, "HE_ASYNC applies to he_matmul_host only");
  if (int r = matmul_checks(c, m, k, n, blk, flags, &si)) return r;
  if (!m || !k || !n) return HE_OK;
  if (!ct_in || !pt || !ct_out || !workspace) return fail(HE_EINVAL, "NULL buffer");
  const u64 need = (flags & HE_DROP_C0) ? si.workspace_bytes_compact : si.workspace_bytes;
  if (workspace_bytes < need) return fail(HE_ENOMEM, "workspace smaller than he_sizes() requires for these flags");
  if (int r = set_device(c)) return r;
  return matmul_device(c, ct_in, pt, m, k, n, blk, 1, mask_seed, flags, ct_out, workspace, (cudaStream_t)stream);
}

int he_matmul_batch(he_ctx* c, const uint64_t* ct_in, const uint64_t* pt, uint32_t m, uint32_t k, uint32_t n,
                    const he_blocking* blk, uint32_t batch, uint64_t mask_seed, uint32_t flags, uint64_t* ct_out,
                    void* workspace, size_t workspace_bytes, void* stream) {
  he_size_info si;
  if (flags & HE_ASYNC) return fail(HE_EINVAL, "HE_ASYNC applies to he_matmul_host only");
  if (int r = matmul_checks(c, m, k, n, blk, flags, &si)) return r;
  if (!m || !k || !n || !batch) return HE_OK;
  if ((u64)batch * c->C.L > 65535) return fail(HE_EINVAL, "batch * L must be <= 65535");
  if (!ct_in || !pt || !ct_out || !workspace) return fail(HE_EINVAL, "NULL buffer");
  const u64 need = (flags & HE_DROP_C0) ? si.workspace_bytes_compact : si.workspace_bytes;
  if (workspace_bytes / batch < need)
    return fail(HE_ENOMEM, "workspace smaller than batch x what he_sizes() requires for these flags");
  if (int r = set_device(c)) return r;
  return matmul_device(c, ct_in, pt, m, k, n, blk, batch, mask_seed, flags, ct_out, workspace, (cudaStream_t)stream);
}

int he_autotune_blocking(he_ctx* c, uint32_t m, uint32_t k, uint32_t n, uint32_t weights_per_call, uint32_t flags,
                         uint32_t batch, uint32_t candidates, void* scratch, size_t scratch_bytes,
                         size_t* scratch_needed, he_blocking* out, float* best_ms, void* stream) {
  if (!c || !out) return fail(HE_EINVAL, "NULL argument");
  if (flags & ~(uint32_t)HE_DROP_C0) return fail(HE_EINVAL, "flags other than HE_DROP_C0");
  if ((u64)(batch ? batch : 1) * c->C.L > 65535) return fail(HE_EINVAL, "batch * L must be <= 65535");
  batch = batch ? batch : 1;
  candidates = candidates ? std::min(candidates, 16u) : 6u;
  std::vector<Candidate> all = blocking_candidates(c->C.N, c->C.L, m, k, n, weights_per_call, c->mac_engine);
  std::vector<he_blocking> cand;
  for (const Candidate& x : all) {
    if ((flags & HE_DROP_C0) && !pow2(x.b.k_b)) continue;
    cand.push_back(x.b);
    if (cand.size() == candidates) break;
  }
  if (cand.empty()) return fail(HE_EINVAL, "no blocking fits");
  *out = cand.front();
  if (best_ms) *best_ms = 0.f;
  if (!m || !k || !n) return HE_OK;
  // scratch: [W: batch k n][pt][ct_in][ct_out][workspace], each 256-byte aligned
  auto up = [](u64 b) { return (b + 255) & ~(u64)255; };
  struct Parts { u64 w, pt, in, out, ws; };
  auto parts = [&](const he_blocking& b) {
    he_size_info si;
    he_sizes(c, m, k, n, &b, &si);
    const bool compact = flags & HE_DROP_C0;
    return Parts{up(8ull * batch * k * n), up(8ull * batch * si.pt_words), up(8ull * batch * si.in_words),
                 up(8ull * batch * (compact ? si.out_words_compact : si.out_words)),
                 up((u64)batch * (compact ? si.workspace_bytes_compact : si.workspace_bytes))};
  };
  u64 need = 0;
  for (const he_blocking& b : cand) {
    const Parts p = parts(b);
    need = std::max(need, p.w + p.pt + p.in + p.out + p.ws);
  }
  if (scratch_needed) *scratch_needed = need;
  if (!scratch) return HE_OK;
  if (scratch_bytes < need) return fail(HE_ENOMEM, "scratch smaller than *scratch_needed");
  if (int r = set_device(c)) return r;
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t e0 = get_event(c), e1 = get_event(c);
  float best = -1.f;
  int rc = HE_OK;
  for (size_t ci = 0; ci < cand.size() && rc == HE_OK; ++ci) {
    const he_blocking& b = cand[ci];
    const Parts p = parts(b);
    uint8_t* base = (uint8_t*)scratch;
    u64* W = (u64*)base;
    u64* pt = (u64*)(base + p.w);
    u64* ct = (u64*)(base + p.w + p.pt);
    u64* o = (u64*)(base + p.w + p.pt + p.in);
    void* ws = base + p.w + p.pt + p.in + p.out;
    Shape s = shape_of(m, k, n, &b);
    auto encode = [&] {
      if (use_coset(c, &b))
        return launch(c, KCosetEnc, st, "autotune: encode (cosets)", [&] {
          return he::launch_coset_encode_weights(c->C, W, k, n, to_blk(&b), s.nI, s.nJ, batch, use_tcr(c, &b, s.nJ), pt,
                                                 st);
        });
      return launch(c, KEncode, st, "autotune: encode", [&] {
        return he::launch_encode_weights(c->C, W, k, n, to_blk(&b), s.nI, s.nJ, batch, use_tc(c, &b, s.nJ), pt, st);
      });
    };
    if ((rc = launch(c, KProbe, st, "autotune: fill", [&] {
           cudaError_t e = he::launch_fill_random(c->C, W, p.w / 8, 0x5eedull, 1, st);
           return e == cudaSuccess ? he::launch_fill_random(c->C, ct, p.in / 8, 0x5eedull + 1, 0, st) : e;
         })))
      break;
    if (!weights_per_call && (rc = encode())) break;
    float cand_best = -1.f;
    for (int rep = 0; rep < 4 && rc == HE_OK; ++rep) {  // one warm-up, three timed
      cudaEventRecord(e0, st);
      if (weights_per_call) rc = encode();
      if (rc == HE_OK) rc = matmul_device(c, ct, pt, m, k, n, &b, batch, 1, flags, o, ws, st);
      cudaEventRecord(e1, st);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep && (cand_best < 0 || ms < cand_best)) cand_best = ms;
    }
    if (rc == HE_OK && (best < 0 || cand_best < best)) {
      best = cand_best;
      *out = b;
    }
  }
  c->pool.push_back(e0);
  c->pool.push_back(e1);
  if (rc != HE_OK) return rc;
  if (int r = he_device_status(c, stream)) return r;
  if (best_ms) *best_ms = best;
  return HE_OK;
}

int he_set_mac_engine(he_ctx* c, uint32_t engine) {
  if (!c) return fail(HE_EINVAL, "ctx is NULL");
  if (engine > HE_MAC_COSET)
    return fail(HE_EINVAL, "engine must be HE_MAC_AUTO, HE_MAC_INTEGER, HE_MAC_TENSOR or HE_MAC_COSET");
  c->mac_engine = engine;
  return HE_OK;
}

int he_get_mac_engine(const he_ctx* c, uint32_t* engine) {
  if (!c || !engine) return fail(HE_EINVAL, "NULL argument");
  *engine = c->mac_engine;
  return HE_OK;
}

int he_mac_uses_tensor_cores(const he_ctx* c, uint32_t k, const he_blocking* blk, uint32_t* yes) {
  if (!c || !yes) return fail(HE_EINVAL, "NULL argument");
  if (int r = check_blk(c, blk)) return r;
  *yes = use_tc(c, blk, shape_of(1, k, 1, blk).nJ) ? 1 : 0;
  return HE_OK;
}

int he_mac_uses_cosets(const he_ctx* c, const he_blocking* blk, uint32_t* yes) {
  if (!c || !yes) return fail(HE_EINVAL, "NULL argument");
  if (int r = check_blk(c, blk)) return r;
  *yes = use_coset(c, blk) ? 1 : 0;
  return HE_OK;
}

int he_set_ntt_radix(he_ctx* c, uint32_t log2_values) {
  if (!c) return fail(HE_EINVAL, "ctx is NULL");
  if (c->C.logN < 9) {  // small rings run the shared-memory transforms, which have no radix
    if (log2_values != (uint32_t)he::kNttLogRDefault) return fail(HE_EINVAL, "N < 512 has only the default radix");
    return HE_OK;
  }
  if (!he::ntt_radix_built(c->C.logN, log2_values)) return fail(HE_EINVAL, "radix not built for this N");
  c->C.logR = log2_values;
  return HE_OK;
}

int he_get_ntt_radix(const he_ctx* c, uint32_t* log2_values) {
  if (!c || !log2_values) return fail(HE_EINVAL, "NULL argument");
  *log2_values = c->C.logR;
  return HE_OK;
}

int he_autotune_ntt_radix(he_ctx* c, uint32_t cnt, void* scratch, size_t scratch_bytes, size_t* scratch_needed,
                          float* ms, uint32_t* chosen, void* stream) {
  if (!c) return fail(HE_EINVAL, "ctx is NULL");
  if (ms)
    for (int i = 0; i < 3; ++i) ms[i] = -1.f;
  if (chosen) *chosen = c->C.logR;
  if (c->C.logN < 9) {  // shared-memory transforms only: nothing to choose
    if (scratch_needed) *scratch_needed = 0;
    return HE_OK;
  }
  const u64 poly_bytes = 8ull * c->C.L * c->C.N;
  if (!cnt) cnt = (uint32_t)std::max<u64>(1, (256ull << 20) / poly_bytes);  // larger than L2
  const u64 need = (u64)cnt * poly_bytes;
  if (scratch_needed) *scratch_needed = need;
  if (!scratch) return HE_OK;
  if (scratch_bytes < need) return fail(HE_ENOMEM, "scratch smaller than *scratch_needed");
  if (int r = set_device(c)) return r;
  cudaStream_t st = (cudaStream_t)stream;
  u64* polys = (u64*)scratch;
  const u64 npolys = (u64)cnt * c->C.L;
  int rc = launch(c, KProbe, st, "autotune radix: fill",
                  [&] { return he::launch_fill_random(c->C, polys, npolys * c->C.N, 0x7adull, 0, st); });
  if (rc) return rc;
  const u32 keep = c->C.logR;
  cudaEvent_t e0 = get_event(c), e1 = get_event(c);
  float best = -1.f, def_ms = -1.f;
  u32 best_r = keep;
  for (u32 r = 3; r <= 5 && rc == HE_OK; ++r) {
    if (!he::ntt_radix_built(c->C.logN, r)) continue;
    c->C.logR = r;
    float rbest = -1.f;
    for (int rep = 0; rep < 4 && rc == HE_OK; ++rep) {  // one warm-up, three timed round trips
      cudaEventRecord(e0, st);
      rc = launch(c, KNttFwd, st, "autotune radix: forward",
                  [&] { return he::launch_ntt_forward(c->C, polys, polys, npolys, st); });
      if (rc == HE_OK)
        rc = launch(c, KNttInv, st, "autotune radix: inverse",
                    [&] { return he::launch_ntt_inverse(c->C, polys, polys, npolys, st); });
      cudaEventRecord(e1, st);
      cudaEventSynchronize(e1);
      float t = 0.f;
      cudaEventElapsedTime(&t, e0, e1);
      if (rep && (rbest < 0 || t < rbest)) rbest = t;
    }
    if (rc != HE_OK) break;
    if (ms) ms[r - 3] = rbest;
    if (r == (u32)he::kNttLogRDefault) def_ms = rbest;
    if (best < 0 || rbest < best) {
      best = rbest;
      best_r = r;
    }
  }
  // The round trips time the transforms alone; inside a layer they share the GPU with the
  // multiply-accumulate.  Measured on GB300 at N = 8192: 8 values per thread 2.4% faster
  // than 16 here, but the BERT-large layer 2% slower with it.  So another radix replaces
  // the default only when it is at least 5% faster.
  if (rc == HE_OK && def_ms > 0 && best > 0.95f * def_ms) best_r = he::kNttLogRDefault;
  c->pool.push_back(e0);
  c->pool.push_back(e1);
  c->C.logR = rc == HE_OK ? best_r : keep;
  if (rc != HE_OK) return rc;
  if (chosen) *chosen = best_r;
  return he_device_status(c, stream);
}

int he_matmul_batch_host(he_ctx* c, const uint64_t* ct_in_host, const uint64_t* pt, uint32_t m, uint32_t k,
                         uint32_t n, const he_blocking* blk, uint32_t batch, uint64_t mask_seed, uint32_t flags,
                         uint64_t* ct_out_host, void* workspace, size_t workspace_bytes, void* stream) {
  he_size_info si;
  if (int r = matmul_checks(c, m, k, n, blk, flags, &si)) return r;
  if (!m || !k || !n || !batch) return HE_OK;
  if ((u64)batch * c->C.L > 65535) return fail(HE_EINVAL, "batch * L must be <= 65535");
  if (!ct_in_host || !pt || !ct_out_host || !workspace) return fail(HE_EINVAL, "NULL buffer");
  const bool compact = flags & HE_DROP_C0;
  const u64 ws_need = (u64)batch * (compact ? si.workspace_bytes_compact : si.workspace_bytes);
  const u64 in_words = (u64)batch * si.in_words, out_words = (u64)batch * (compact ? si.out_words_compact : si.out_words);
  const u64 need = ws_need + 8 * (in_words + out_words);
  if (workspace_bytes < need) return fail(HE_ENOMEM, "workspace smaller than he_matmul_host needs");
  if (int r = set_device(c)) return r;
  cudaStream_t st = (cudaStream_t)stream;
  u64* d_in = (u64*)((char*)workspace + ws_need);
  u64* d_out = d_in + in_words;
  cudaError_t e = cudaMemcpyAsync(d_in, ct_in_host, in_words * 8, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_fail(e, "matmul_host: upload");
  if (int r = matmul_device(c, d_in, pt, m, k, n, blk, batch, mask_seed, flags, d_out, workspace, st)) return r;
  e = cudaMemcpyAsync(ct_out_host, d_out, out_words * 8, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && !(flags & HE_ASYNC)) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "matmul_host: download");
  return HE_OK;
}

int he_matmul_host(he_ctx* c, const uint64_t* ct_in_host, const uint64_t* pt, uint32_t m, uint32_t k, uint32_t n,
                   const he_blocking* blk, uint64_t mask_seed, uint32_t flags, uint64_t* ct_out_host,
                   void* workspace, size_t workspace_bytes, void* stream) {
  return he_matmul_batch_host(c, ct_in_host, pt, m, k, n, blk, 1, mask_seed, flags, ct_out_host, workspace,
                              workspace_bytes, stream);
}

int he_matmul_noalloc(he_ctx* c, const uint64_t* ct_in, const uint64_t* pt, uint32_t m, uint32_t k, uint32_t n,
                      const he_blocking* blk, uint64_t mask_seed, uint32_t flags, uint64_t* ct_out, void* stream) {
  static_assert(HE_NOALLOC_SCRATCH_BYTES == he::kNoAllocScratchBytes, "scratch size mismatch");
  he_size_info si;
  if (int r = matmul_checks(c, m, k, n, blk, flags, &si)) return r;
  if (!m || !k || !n) return HE_OK;
  if (!ct_in || !pt || !ct_out) return fail(HE_EINVAL, "NULL buffer");
  if (flags & HE_ASYNC) return fail(HE_EINVAL, "HE_ASYNC applies to he_matmul_host only");
  const u64 need = (flags & HE_DROP_C0) ? si.workspace_bytes_compact : si.workspace_bytes;
  if (need > HE_NOALLOC_SCRATCH_BYTES)
    return fail(HE_EINVAL, "product needs " + std::to_string(need) + " bytes of scratch; he_matmul_noalloc has " +
                               std::to_string((size_t)HE_NOALLOC_SCRATCH_BYTES) + " (use he_matmul)");
  if (int r = set_device(c)) return r;
  void* scratch = nullptr;
  cudaError_t e = he::noalloc_scratch_address(c->device, &scratch);
  if (e != cudaSuccess) return cuda_fail(e, "matmul_noalloc: scratch address");
  return matmul_device(c, ct_in, pt, m, k, n, blk, 1, mask_seed, flags, ct_out, scratch, (cudaStream_t)stream);
}

// ---------------------------------------------------------------- multi-product launch

namespace {

struct MultiPlan {
  he::MultiTable T;
  u64 fwd = 0, mac = 0, tc = 0, inv = 0, c0 = 0, ws_bytes = 0;
  u64 cfwd = 0, cinv = 0, tcr = 0;  // blocks of the coset grids, units of the row-major MAC (coset products)
  u32 max_nc = 0;  // shared-memory words of the largest c0 transform
};

// Validates the products and lays out the table; workspace may be NULL (size query).
// Compact products (HE_DROP_C0) at N >= 512 that share their encoded weights, k, n and
// blocking become one merged item: their row-blocks back to back, so every weight stage
// of the multiply-accumulate serves all of their rows (requests of one weight matrix in a
// serving batch); each keeps its own inputs, outputs, mask seed and output indices, and
// its result is bit-identical to its own he_matmul call.
int plan_multi(const he_ctx* c, uint32_t count, const he_product* items, char* workspace, MultiPlan* P) {
  if (count > (u32)he::kMaxMulti) return fail(HE_EINVAL, "at most 64 products per multi-product launch");
  if (count && !items) return fail(HE_EINVAL, "items is NULL");
  const u64 N = c->C.N, L = c->C.L;
  const u32 rows_t = he::mac_tile_rows(), cols_t = he::mac_tile_cols();
  auto same_blk = [](const he_blocking& a, const he_blocking& b) {
    return a.m_b == b.m_b && a.k_b == b.k_b && a.n_b == b.n_b;
  };
  std::vector<std::vector<u32>> groups;  // products of each launch item, in first-appearance order
  for (u32 i = 0; i < count; ++i) {
    const he_product& x = items[i];
    if (int r = check_blk(c, &x.blk)) return r;
    if (x.flags & ~(uint32_t)(HE_DROP_C0 | HE_SEED_DEVICE)) return fail(HE_EINVAL, "unknown flags");
    if ((x.flags & HE_SEED_DEVICE) && !x.mask_seed) return fail(HE_EINVAL, "HE_SEED_DEVICE with a NULL seed address");
    const bool compact = x.flags & HE_DROP_C0;
    if (compact && !pow2(x.blk.k_b)) return fail(HE_EINVAL, "HE_DROP_C0 needs a power-of-two k_b");
    if (!x.m || !x.k || !x.n) continue;
    if (!x.ct_in || !x.pt || !x.ct_out) return fail(HE_EINVAL, "NULL buffer in a product");
    if (shape_of(x.m, x.k, x.n, &x.blk).nJ > 4096) return fail(HE_EINVAL, "at most 4096 k-blocks per product");
    bool placed = false;
    if (compact && c->C.logN >= 9) {
      for (auto& g : groups) {
        const he_product& y = items[g[0]];
        if ((y.flags & HE_DROP_C0) && y.pt == x.pt && y.k == x.k && y.n == x.n && same_blk(y.blk, x.blk)) {
          g.push_back(i);
          placed = true;
          break;
        }
      }
    }
    if (!placed) groups.push_back({i});
  }
  P->T.count = 0;
  P->T.nseg = 0;
  u64 off = 0;
  auto take = [&](u64 bytes) -> u64* {
    off = (off + 255) & ~(u64)255;
    u64* ptr = workspace ? (u64*)(workspace + off) : nullptr;
    off += bytes;
    return ptr;
  };
  for (const auto& g : groups) {
    const he_product& x = items[g[0]];
    const bool compact = x.flags & HE_DROP_C0;
    Shape s = shape_of(x.m, x.k, x.n, &x.blk);
    he::MultiItem& it = P->T.it[P->T.count++];
    memset(&it, 0, sizeof(it));
    it.pt = x.pt;
    if (g.size() == 1) {
      it.ct_in = x.ct_in;
      it.out = x.ct_out;
      it.mask_seed = x.mask_seed;
      it.seed_dev = (x.flags & HE_SEED_DEVICE) ? reinterpret_cast<const u64*>((uintptr_t)x.mask_seed) : nullptr;
    } else {
      it.seg0 = P->T.nseg;
      it.nseg = (u32)g.size();
      u32 lb = 0;
      for (u32 i : g) {
        const he_product& y = items[i];
        he::MultiSeg& sg = P->T.seg[P->T.nseg++];
        sg.ct_in = y.ct_in;
        sg.out = y.ct_out;
        sg.mask_seed = y.mask_seed;
        sg.seed_dev = (y.flags & HE_SEED_DEVICE) ? reinterpret_cast<const u64*>((uintptr_t)y.mask_seed) : nullptr;
        sg.lb0 = lb;
        sg.pad = 0;
        lb += shape_of(y.m, y.k, y.n, &y.blk).nLb;
      }
      s.nLb = lb;
    }
    it.fwd_begin = P->fwd;
    it.mac_begin = P->mac;
    it.inv_begin = P->inv;
    it.c0_begin = P->c0;
    if (use_coset(c, &x.blk)) {  // forward, multiply-accumulate and inverse in the coset grids
      const CosetGeom cg = coset_geom(c, &x.blk, s.nI, s.nJ, s.nLb);
      u64* ws = take(up256(cg.ctn_words * 8) + cg.acc_words * 8);
      coset_item(c, it, &x.blk, s, compact, ws, &P->cfwd, &P->tc, &P->tcr, &P->cinv);
      continue;
    }
    it.cfwd_begin = P->cfwd;
    it.cinv_begin = P->cinv;
    it.tcr_begin = P->tcr;
    it.nI = s.nI;
    it.nJ = s.nJ;
    it.nLb = s.nLb;
    it.compact = compact;
    it.logkb = compact ? log2u(x.blk.k_b) : 0;
    it.tilesR = (2 * s.nLb + rows_t - 1) / rows_t;
    it.tilesC = (s.nI + cols_t - 1) / cols_t;
    it.tc = use_tc(c, &x.blk, s.nJ);
    const u64 out_cts = (u64)s.nLb * s.nI;
    it.ctN = take(operand_words(c, &x.blk, 2 * s.nLb, s.nJ) * 8);
    if (compact) {
      it.c0_ntt = take(out_cts * L * N * 8);
      P->max_nc = std::max<u32>(P->max_nc, he::c0_smem_words((u32)N, it.logkb));
    }
    if (it.nseg) it.c1_ntt = take(out_cts * L * N * 8);
    it.fwd_begin = P->fwd;
    it.mac_begin = P->mac;
    it.inv_begin = P->inv;
    it.c0_begin = P->c0;
    it.tc_begin = P->tc;
    P->fwd += (u64)s.nLb * s.nJ * 2 * L;
    if (it.tc) P->tc += he::tc_units((u32)N, (u32)L, s.nI, 2 * s.nLb);
    else P->mac += (N >> 5) * it.tilesR * it.tilesC * L;
    P->inv += out_cts * (compact ? 1 : 2) * L;
    P->c0 += compact ? out_cts * L : 0;
  }
  P->ws_bytes = off;
  if (P->fwd >= (1ull << 31) || P->mac >= (1ull << 31) || P->tc >= (1ull << 31) || P->inv >= (1ull << 31) ||
      P->cfwd >= (1ull << 31) || P->cinv >= (1ull << 31) || P->tcr >= (1ull << 31))
    return fail(HE_EINVAL, "multi-product launch too large");
  return HE_OK;
}

}  // namespace

int he_multi_workspace_bytes(const he_ctx* c, uint32_t count, const he_product* items, size_t* bytes) {
  if (!c || !bytes) return fail(HE_EINVAL, "NULL argument");
  MultiPlan P;
  if (int r = plan_multi(c, count, items, nullptr, &P)) return r;
  *bytes = P.ws_bytes;
  return HE_OK;
}

int he_matmul_multi(he_ctx* c, uint32_t count, const he_product* items, void* workspace, size_t workspace_bytes,
                    void* stream) {
  if (!c) return fail(HE_EINVAL, "ctx is NULL");
  MultiPlan P;
  if (int r = plan_multi(c, count, items, (char*)workspace, &P)) return r;
  if (!P.T.count) return HE_OK;
  if (!workspace) return fail(HE_EINVAL, "workspace is NULL");
  if (workspace_bytes < P.ws_bytes) return fail(HE_ENOMEM, "workspace smaller than he_multi_workspace_bytes()");
  if (int r = set_device(c)) return r;
  cudaStream_t st = (cudaStream_t)stream;
  int r = HE_OK;
  if (P.fwd)
    r = launch(c, KNttFwd, st, "multi: forward NTT", [&] { return he::launch_fwd_multi(c->C, P.T, P.fwd, st); });
  if (!r && P.cfwd)
    r = launch(c, KCosetFwd, st, "multi: coset forward transforms",
               [&] { return he::launch_coset_fwd_multi(c->C, P.T, P.cfwd, st); });
  if (!r && P.mac)
    r = launch(c, KMac, st, "multi: multiply-accumulate",
               [&] { return he::launch_mac_multi(c->C, P.T, P.mac, c->d_err, st); });
  if (!r && P.tc)
    r = launch(c, KMacTc, st, "multi: tensor-core multiply-accumulate",
               [&] { return he::launch_mac_tc_multi(c->C, P.T, P.tc, c->d_err, st); });
  if (!r && P.tcr)
    r = launch(c, KMacTc, st, "multi: row-major tensor-core multiply-accumulate",
               [&] { return he::launch_mac_tcr_multi(c->C, P.T, P.tcr, c->d_err, st); });
  if (!r && P.c0) {  // compact products: c1 inverse NTTs and pruned c0 transforms in one grid
    r = launch(c, KInvC0, st, "multi: inverse NTT of c1 + pruned inverse NTT of c0",
               [&] { return he::launch_inv_c0_multi(c->C, P.T, P.inv, P.c0, P.max_nc, st); });
    if (!r && !he::inv_c0_fused(c->C)) c->launches.fetch_add(1, std::memory_order_relaxed);  // two grids there
  } else if (!r && P.inv) {
    r = launch(c, KInttMask, st, "multi: inverse NTT", [&] { return he::launch_inv_multi(c->C, P.T, P.inv, st); });
  }
  if (!r && P.cinv)
    r = launch(c, KCosetInv, st, "multi: coset inverse transforms + mask",
               [&] { return he::launch_coset_inv_multi(c->C, P.T, P.cinv, st); });
  return r;
}

namespace {

// Device words of one product's input and output ciphertexts (output compact with DROP_C0).
void product_io_words(const he_ctx* c, const he_product& x, u64* in_w, u64* out_w) {
  he_size_info si;
  he_sizes(c, x.m, x.k, x.n, &x.blk, &si);
  const bool empty = !x.m || !x.k || !x.n;
  *in_w = empty ? 0 : si.in_words;
  *out_w = empty ? 0 : ((x.flags & HE_DROP_C0) ? si.out_words_compact : si.out_words);
}

}  // namespace

int he_multi_host_workspace_bytes(const he_ctx* c, uint32_t count, const he_product* items, size_t* bytes) {
  if (!c || !bytes) return fail(HE_EINVAL, "NULL argument");
  MultiPlan P;
  if (int r = plan_multi(c, count, items, nullptr, &P)) return r;
  u64 need = up256(P.ws_bytes);
  for (u32 i = 0; i < count; ++i) {
    u64 in_w, out_w;
    product_io_words(c, items[i], &in_w, &out_w);
    need += up256(8 * in_w) + up256(8 * out_w);
  }
  *bytes = need;
  return HE_OK;
}

int he_matmul_multi_host(he_ctx* c, uint32_t count, const he_product* items, uint32_t flags, void* workspace,
                         size_t workspace_bytes, void* stream) {
  if (!c) return fail(HE_EINVAL, "ctx is NULL");
  if (flags & ~(uint32_t)HE_ASYNC) return fail(HE_EINVAL, "flags other than HE_ASYNC");
  size_t need = 0;
  if (int r = he_multi_host_workspace_bytes(c, count, items, &need)) return r;
  if (!count) return HE_OK;
  if (!workspace) return fail(HE_EINVAL, "workspace is NULL");
  if (workspace_bytes < need) return fail(HE_ENOMEM, "workspace smaller than he_multi_host_workspace_bytes()");
  MultiPlan P;
  if (int r = plan_multi(c, count, items, nullptr, &P)) return r;
  if (int r = set_device(c)) return r;
  cudaStream_t st = (cudaStream_t)stream;
  // [multi-product workspace][inputs][outputs]: the items' host buffers staged on the device
  std::vector<he_product> dev(items, items + count);
  char* base = (char*)workspace;
  u64 off = up256(P.ws_bytes);
  for (u32 i = 0; i < count; ++i) {
    u64 in_w, out_w;
    product_io_words(c, items[i], &in_w, &out_w);
    if (in_w && (!items[i].ct_in || !items[i].ct_out)) return fail(HE_EINVAL, "NULL host buffer");
    dev[i].ct_in = (const uint64_t*)(base + off);
    off += up256(8 * in_w);
    dev[i].ct_out = (uint64_t*)(base + off);
    off += up256(8 * out_w);
    if (in_w) {
      cudaError_t e = cudaMemcpyAsync((void*)dev[i].ct_in, items[i].ct_in, 8 * in_w, cudaMemcpyHostToDevice, st);
      if (e != cudaSuccess) return cuda_fail(e, "matmul_multi_host: upload");
    }
  }
  if (int r = he_matmul_multi(c, count, dev.data(), workspace, P.ws_bytes, stream)) return r;
  for (u32 i = 0; i < count; ++i) {
    u64 in_w, out_w;
    product_io_words(c, items[i], &in_w, &out_w);
    if (!out_w) continue;
    cudaError_t e = cudaMemcpyAsync(items[i].ct_out, dev[i].ct_out, 8 * out_w, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return cuda_fail(e, "matmul_multi_host: download");
  }
  if (!(flags & HE_ASYNC)) {
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "matmul_multi_host: synchronize");
  }
  return HE_OK;
}

}  // extern "C"

struct he_pipe {
  he_ctx* c = nullptr;
  uint32_t depth = 0;
  uint64_t submits = 0;
  cudaStream_t up = nullptr, comp = nullptr, down = nullptr;
  std::vector<cudaEvent_t> uploaded, computed, downloaded;  // per slot
};

extern "C" {

int he_pipe_create(he_ctx* c, uint32_t depth, he_pipe** out) {
  if (!c || !out) return fail(HE_EINVAL, "NULL argument");
  if (!depth || depth > 16) return fail(HE_EINVAL, "pipe depth must be 1 .. 16");
  if (int r = set_device(c)) return r;
  he_pipe* p = new he_pipe;
  p->c = c;
  p->depth = depth;
  cudaError_t e = cudaSuccess;
  for (cudaStream_t* s : {&p->up, &p->comp, &p->down})
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(s, cudaStreamNonBlocking);
  for (auto* v : {&p->uploaded, &p->computed, &p->downloaded})
    for (uint32_t i = 0; i < depth && e == cudaSuccess; ++i) {
      cudaEvent_t ev = nullptr;
      e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
      if (e == cudaSuccess) v->push_back(ev);
    }
  if (e != cudaSuccess) {
    he_pipe_free(p);
    return cuda_fail(e, "pipe_create");
  }
  *out = p;
  return HE_OK;
}

int he_pipe_free(he_pipe* p) {
  if (!p) return HE_OK;
  set_device(p->c);
  for (cudaStream_t s : {p->up, p->comp, p->down})
    if (s) cudaStreamSynchronize(s);
  for (auto* v : {&p->uploaded, &p->computed, &p->downloaded})
    for (cudaEvent_t ev : *v) cudaEventDestroy(ev);
  for (cudaStream_t s : {p->up, p->comp, p->down})
    if (s) cudaStreamDestroy(s);
  delete p;
  return HE_OK;
}

int he_pipe_compute_stream(he_pipe* p, void** stream) {
  if (!p || !stream) return fail(HE_EINVAL, "NULL argument");
  *stream = (void*)p->comp;
  return HE_OK;
}

}  // extern "C"

namespace {

constexpr uint32_t kPipeChunk = 64;  // products per multi-product launch

// One copy per run of consecutive products whose source buffers and destination buffers
// are both adjacent (8 * words[i] bytes each, empty products skipped): the host link moves
// a few large copies much faster than one per product.  Adjacent host buffers may still
// belong to different allocations (two pinned arrays side by side), which one copy may
// not span: the runtime then rejects the copy at enqueue time (nothing is queued), the
// error is cleared and the run goes product by product.
template <class Dst, class Src>
cudaError_t copy_runs(uint32_t count, const u64* words, Dst dst, Src src, cudaMemcpyKind kind, cudaStream_t st) {
  uint32_t i = 0;
  while (i < count) {
    if (!words[i]) {
      ++i;
      continue;
    }
    char* d0 = dst(i);
    const char* s0 = src(i);
    u64 bytes = 8 * words[i];
    uint32_t j = i + 1;
    for (; j < count && words[j] && dst(j) == d0 + bytes && src(j) == s0 + bytes; ++j) bytes += 8 * words[j];
    cudaError_t e = cudaMemcpyAsync(d0, s0, bytes, kind, st);
    if (e == cudaErrorInvalidValue && j > i + 1) {
      cudaGetLastError();  // not sticky: clear it so later checks do not see it
      e = cudaSuccess;
      for (uint32_t k = i; k < j && e == cudaSuccess; ++k) e = cudaMemcpyAsync(dst(k), src(k), 8 * words[k], kind, st);
    }
    if (e != cudaSuccess) return e;
    i = j;
  }
  return cudaSuccess;
}

// Bytes of one pipe slot: the largest chunk's multi-product workspace, then every
// product's staged input and output.
int pipe_slot_bytes(he_ctx* c, uint32_t count, const he_product* items, u64* bytes) {
  u64 ws = 0, io = 0;
  for (uint32_t i0 = 0; i0 < count; i0 += kPipeChunk) {
    MultiPlan P;
    if (int r = plan_multi(c, std::min(kPipeChunk, count - i0), items + i0, nullptr, &P)) return r;
    ws = std::max(ws, (u64)P.ws_bytes);
  }
  for (uint32_t i = 0; i < count; ++i) {
    u64 in_w, out_w;
    product_io_words(c, items[i], &in_w, &out_w);
    io += up256(8 * in_w) + up256(8 * out_w);
  }
  *bytes = up256(ws) + io;
  return HE_OK;
}

}  // namespace

extern "C" {

int he_pipe_workspace_bytes(const he_pipe* p, uint32_t count, const he_product* items, size_t* bytes) {
  if (!p || !bytes || (count && !items)) return fail(HE_EINVAL, "NULL argument");
  u64 slot = 0;
  if (int r = pipe_slot_bytes(p->c, count, items, &slot)) return r;
  *bytes = (size_t)p->depth * slot;
  return HE_OK;
}

int he_pipe_submit(he_pipe* p, uint32_t count, const he_product* items, void* workspace, size_t workspace_bytes) {
  if (!p) return fail(HE_EINVAL, "pipe is NULL");
  if (!count) return HE_OK;
  if (!items) return fail(HE_EINVAL, "items is NULL");
  he_ctx* c = p->c;
  u64 need = 0;
  if (int r = pipe_slot_bytes(c, count, items, &need)) return r;
  if (!workspace) return fail(HE_EINVAL, "workspace is NULL");
  const u64 slot_bytes = (workspace_bytes / p->depth) & ~(u64)255;
  if (slot_bytes < need) return fail(HE_ENOMEM, "workspace smaller than he_pipe_workspace_bytes()");
  if (int r = set_device(c)) return r;
  const uint32_t slot = (uint32_t)(p->submits % p->depth);
  const bool reuse = p->submits >= p->depth;
  char* base = (char*)workspace + slot * slot_bytes;
  u64 ws = 0;
  for (uint32_t i0 = 0; i0 < count; i0 += kPipeChunk) {
    MultiPlan P;
    if (int r = plan_multi(c, std::min(kPipeChunk, count - i0), items + i0, nullptr, &P)) return r;
    ws = std::max(ws, (u64)P.ws_bytes);
  }
  // slot: [multi-product workspace][every input][every output], so that products whose
  // host buffers are adjacent (e.g. slices of one array) move in one copy
  std::vector<he_product> dev(items, items + count);
  std::vector<u64> in_words(count), out_words(count);
  u64 off = up256(ws);
  for (u32 i = 0; i < count; ++i) {
    product_io_words(c, items[i], &in_words[i], &out_words[i]);
    if (in_words[i] && (!items[i].ct_in || !items[i].ct_out)) return fail(HE_EINVAL, "NULL host buffer");
    dev[i].ct_in = (const uint64_t*)(base + off);
    off += up256(8 * in_words[i]);
  }
  for (u32 i = 0; i < count; ++i) {
    dev[i].ct_out = (uint64_t*)(base + off);
    off += up256(8 * out_words[i]);
  }
  cudaError_t e = cudaSuccess;
  // uploads: after the launches that last read this slot
  if (reuse) e = cudaStreamWaitEvent(p->up, p->computed[slot], 0);
  if (e == cudaSuccess)
    e = copy_runs(count, in_words.data(), [&](u32 i) { return (char*)dev[i].ct_in; },
                  [&](u32 i) { return (char*)items[i].ct_in; }, cudaMemcpyHostToDevice, p->up);
  if (e == cudaSuccess) e = cudaEventRecord(p->uploaded[slot], p->up);
  // launches: after the uploads and after the downloads that last read this slot's outputs
  if (e == cudaSuccess) e = cudaStreamWaitEvent(p->comp, p->uploaded[slot], 0);
  if (e == cudaSuccess && reuse) e = cudaStreamWaitEvent(p->comp, p->downloaded[slot], 0);
  if (e != cudaSuccess) return cuda_fail(e, "pipe_submit: upload");
  for (uint32_t i0 = 0; i0 < count; i0 += kPipeChunk)
    if (int r = he_matmul_multi(c, std::min(kPipeChunk, count - i0), dev.data() + i0, base, ws, (void*)p->comp))
      return r;
  e = cudaEventRecord(p->computed[slot], p->comp);
  // downloads: after the launches
  if (e == cudaSuccess) e = cudaStreamWaitEvent(p->down, p->computed[slot], 0);
  if (e == cudaSuccess)
    e = copy_runs(count, out_words.data(), [&](u32 i) { return (char*)items[i].ct_out; },
                  [&](u32 i) { return (char*)dev[i].ct_out; }, cudaMemcpyDeviceToHost, p->down);
  if (e == cudaSuccess) e = cudaEventRecord(p->downloaded[slot], p->down);
  if (e != cudaSuccess) return cuda_fail(e, "pipe_submit: download");
  ++p->submits;
  return HE_OK;
}

int he_pipe_wait(he_pipe* p) {
  if (!p) return fail(HE_EINVAL, "pipe is NULL");
  if (int r = set_device(p->c)) return r;
  cudaError_t e = cudaStreamSynchronize(p->down);  // the downloads wait on every other queue
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->comp);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->up);
  return e == cudaSuccess ? HE_OK : cuda_fail(e, "pipe_wait");
}

int he_expand_compact(he_ctx* c, const uint64_t* ct_compact, uint32_t cnt, uint32_t k_b, uint64_t* ct_full,
                      void* stream) {
  if (!c) return fail(HE_EINVAL, "ctx is NULL");
  if (!pow2(k_b) || k_b > c->C.N) return fail(HE_EINVAL, "k_b must be a power of two <= N");
  if (!cnt) return HE_OK;
  if (!ct_compact || !ct_full) return fail(HE_EINVAL, "NULL buffer");
  if (int r = set_device(c)) return r;
  return launch(c, KExpand, (cudaStream_t)stream, "expand_compact", [&] {
    return he::launch_expand_compact(c->C, ct_compact, cnt, log2u(k_b), ct_full, (cudaStream_t)stream);
  });
}

// Words of cnt wire-format ciphertexts: full (k_b = 0) or compact (HE_DROP_C0 output of
// a product with this power-of-two k_b); logkb receives log2 k_b (0 for full).
static int wire_words(const he_ctx* c, uint32_t cnt, uint32_t k_b, u64* words, u32* logkb) {
  if (k_b && !pow2(k_b)) return fail(HE_EINVAL, "k_b must be 0 (full ciphertexts) or a power of two");
  if (k_b > c->C.N) return fail(HE_EINVAL, "k_b must be at most N");
  *logkb = k_b ? log2u(k_b) : 0;
  *words = (u64)cnt * c->C.L * ((u64)(c->C.N >> *logkb) + c->C.N);
  return HE_OK;
}

int he_ct_export(he_ctx* c, const uint64_t* ct, uint32_t cnt, uint32_t k_b, uint64_t* host_buf, void* stream) {
  if (!c) return fail(HE_EINVAL, "ctx is NULL");
  u64 words;
  u32 logkb;
  if (int r = wire_words(c, cnt, k_b, &words, &logkb)) return r;
  if (!words) return HE_OK;
  if (!ct || !host_buf) return fail(HE_EINVAL, "NULL buffer");
  if (int r = set_device(c)) return r;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(host_buf, ct, words * sizeof(u64), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e == cudaSuccess ? HE_OK : cuda_fail(e, "ct_export: copy to host");
}

int he_ct_import(he_ctx* c, const uint64_t* host_buf, uint32_t cnt, uint32_t k_b, uint64_t* ct, void* stream) {
  if (!c) return fail(HE_EINVAL, "ctx is NULL");
  u64 words;
  u32 logkb;
  if (int r = wire_words(c, cnt, k_b, &words, &logkb)) return r;
  if (!words) return HE_OK;
  if (!ct || !host_buf) return fail(HE_EINVAL, "NULL buffer");
  if (int r = set_device(c)) return r;
  cudaStream_t st = (cudaStream_t)stream;
  u64 bad[2] = {0, ~0ull};
  cudaError_t e = cudaMemcpyAsync(ct, host_buf, words * sizeof(u64), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_bad, bad, sizeof(bad), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_fail(e, "ct_import: copy to device");
  int r = launch(c, KCheck, st, "ct_import: residue check",
                 [&] { return he::launch_check_residues(c->C, ct, cnt, logkb, c->d_bad, st); });
  if (r) return r;
  e = cudaMemcpyAsync(bad, c->d_bad, sizeof(bad), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "ct_import: residue check readback");
  if (bad[0]) {
    const u64 N = c->C.N, L = c->C.L, Nc = N >> logkb, per = L * (Nc + N), w = bad[1] % per;
    const bool c0 = w < L * Nc;
    const u64 l = c0 ? w / Nc : (w - L * Nc) / N;
    return fail(HE_EINVAL, std::to_string(bad[0]) + " word(s) not below their prime; first at word " +
                               std::to_string(bad[1]) + " (ciphertext " + std::to_string(bad[1] / per) +
                               (c0 ? ", c0" : ", c1") + ", prime " + std::to_string(l) + ")");
  }
  return HE_OK;
}

int he_ntt_forward(he_ctx* c, uint64_t* polys, uint32_t cnt, void* stream) {
  if (!c) return fail(HE_EINVAL, "ctx is NULL");
  if (!cnt) return HE_OK;
  if (!polys) return fail(HE_EINVAL, "NULL buffer");
  if (int r = set_device(c)) return r;
  return launch(c, KNttFwd, (cudaStream_t)stream, "ntt_forward", [&] {
    return he::launch_ntt_forward(c->C, polys, polys, (u64)cnt * c->C.L, (cudaStream_t)stream);
  });
}

int he_ntt_inverse(he_ctx* c, uint64_t* polys, uint32_t cnt, void* stream) {
  if (!c) return fail(HE_EINVAL, "ctx is NULL");
  if (!cnt) return HE_OK;
  if (!polys) return fail(HE_EINVAL, "NULL buffer");
  if (int r = set_device(c)) return r;
  return launch(c, KNttInv, (cudaStream_t)stream, "ntt_inverse", [&] {
    return he::launch_ntt_inverse(c->C, polys, polys, (u64)cnt * c->C.L, (cudaStream_t)stream);
  });
}

int he_poly_mul(he_ctx* c, const uint64_t* a, const uint64_t* b, uint64_t* out, uint32_t cnt, void* stream) {
  if (!c) return fail(HE_EINVAL, "ctx is NULL");
  if (!cnt) return HE_OK;
  if (!a || !b || !out) return fail(HE_EINVAL, "NULL buffer");
  if (int r = set_device(c)) return r;
  return launch(c, KPolyMul, (cudaStream_t)stream, "poly_mul", [&] {
    return he::launch_poly_mul(c->C, a, b, out, (u64)cnt * c->C.L, (cudaStream_t)stream);
  });
}

int he_gauss_cdt(uint64_t* out, uint32_t cap) {
  static const uint64_t table[2 * he::kGaussBound] = {
#include "gauss_cdt.inc"
  };
  if (!out || cap < 2 * he::kGaussBound) return fail(HE_EINVAL, "need room for 38 words");
  memcpy(out, table, sizeof(table));
  return HE_OK;
}

int he_profile_enable(he_ctx* c, int on) {
  if (!c) return fail(HE_EINVAL, "ctx is NULL");
  c->prof = on != 0;
  for (auto& r : c->recs) {
    c->pool.push_back(r.e0);
    c->pool.push_back(r.e1);
  }
  c->recs.clear();
  for (int i = 0; i < KCount; ++i) {
    c->stat_launches[i] = 0;
    c->stat_ms[i] = 0;
  }
  return HE_OK;
}

int he_profile_read(he_ctx* c, he_kernel_stat* out, uint32_t cap, uint32_t* n) {
  if (!c || !n) return fail(HE_EINVAL, "NULL argument");
  if (int r = set_device(c)) return r;
  for (auto& r : c->recs) {
    cudaError_t e = cudaEventSynchronize(r.e1);
    if (e != cudaSuccess) return cuda_fail(e, "profile: event sync");
    float ms = 0;
    cudaEventElapsedTime(&ms, r.e0, r.e1);
    c->stat_launches[r.kind] += 1;
    c->stat_ms[r.kind] += ms;
    c->pool.push_back(r.e0);
    c->pool.push_back(r.e1);
  }
  c->recs.clear();
  u32 cnt = 0;
  for (int i = 0; i < KCount; ++i) {
    if (!c->stat_launches[i]) continue;
    if (out && cnt < cap) {
      memset(&out[cnt], 0, sizeof(he_kernel_stat));
      strncpy(out[cnt].name, kKindNames[i], sizeof(out[cnt].name) - 1);
      out[cnt].launches = c->stat_launches[i];
      out[cnt].total_ms = c->stat_ms[i];
    }
    ++cnt;
  }
  *n = cnt;
  return HE_OK;
}

int he_device_status(he_ctx* c, void* stream) {
  if (!c) return fail(HE_EINVAL, "ctx is NULL");
  if (int r = set_device(c)) return r;
  int flag = 0;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(&flag, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess && flag) e = cudaMemsetAsync(c->d_err, 0, sizeof(int), st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "device status readback");
  return flag ? fail(HE_ETIMEOUT, "a kernel's bounded wait for its data expired; results of that call are invalid")
              : HE_OK;
}

int he_probe_tensor(he_ctx* c, uint32_t kind, double* ops_per_s, uint32_t* scratch, size_t scratch_words,
                    void* stream) {
  if (!c || !ops_per_s || !scratch) return fail(HE_EINVAL, "NULL argument");
  if (kind > 1) return fail(HE_EINVAL, "kind must be 0 (tcgen05 bf16) or 1 (mma.sync s8)");
  if (int r = set_device(c)) return r;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
  if ((u64)4 * sms > scratch_words) return fail(HE_EINVAL, "scratch needs 4 x SMs words");
  float ms = 0;
  int iters = 0;
  cudaError_t e = he::probe_tensor((int)kind, sms, c->d_err, scratch, &ms, &iters, (cudaStream_t)stream);
  c->launches.fetch_add(3, std::memory_order_relaxed);
  if (e != cudaSuccess) return cuda_fail(e, "probe_tensor");
  const double ops = kind == 0 ? 2.0 * 128 * 256 * 16 * iters * 2.0 * sms            // per block: iters MMAs
                               : 2.0 * 16 * 8 * 32 * 8.0 * iters * 8.0 * 4.0 * sms;  // 8 warps x 8 chains
  *ops_per_s = ms > 0 ? ops / (ms * 1e-3) : 0.0;
  return HE_OK;
}

int he_test_tc_gemm(he_ctx* c, uint32_t n, uint32_t k, const void* A, const void* B, void* D, void* stream) {
  if (!c || !A || !B || !D) return fail(HE_EINVAL, "NULL argument");
  if (n < 16 || n > 256 || n % 16) return fail(HE_EINVAL, "n must be a multiple of 16 in [16, 256]");
  if (!k || k % 16) return fail(HE_EINVAL, "k must be a positive multiple of 16");
  if ((u64)(128 + n) * k * 2 > 200 * 1024) return fail(HE_EINVAL, "operands exceed 200 KB of shared memory");
  if (int r = set_device(c)) return r;
  return launch(c, KProbe, (cudaStream_t)stream, "tc_gemm check",
                [&] { return he::launch_tc_check(A, B, D, n, k, c->d_err, (cudaStream_t)stream); });
}

int he_probe_mad_wide(he_ctx* c, uint64_t* scratch, size_t scratch_words, double* ops_per_s, double* per_sm_per_clock,
                      void* stream) {
  if (!c || !scratch || !ops_per_s) return fail(HE_EINVAL, "NULL argument");
  if (int r = set_device(c)) return r;
  int sms = 0, clk_khz = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
  cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, c->device);
  if ((u64)sms * 8 * 256 > scratch_words) return fail(HE_EINVAL, "scratch needs SMs x 2048 words");
  float ms = 0;
  cudaError_t e = he::probe_mad_wide(sms, scratch, &ms, (cudaStream_t)stream);
  c->launches.fetch_add(2, std::memory_order_relaxed);
  if (e != cudaSuccess) return cuda_fail(e, "probe_mad_wide");
  const double ops = (double)sms * 8 * 256 * 2048 * 64;
  *ops_per_s = ops / (ms * 1e-3);
  if (per_sm_per_clock) *per_sm_per_clock = *ops_per_s / sms / (clk_khz * 1e3);
  return HE_OK;
}

int he_test_wait_timeout(he_ctx* c, uint32_t limit_ms, void* stream) {
  if (!c) return fail(HE_EINVAL, "ctx is NULL");
  if (!limit_ms || limit_ms > 2000) return fail(HE_EINVAL, "limit_ms must be in [1, 2000]");
  if (int r = set_device(c)) return r;
  return launch(c, KProbe, (cudaStream_t)stream, "wait timeout check", [&] {
    return he::launch_wait_timeout_check((uint64_t)limit_ms * 1000000ull, c->d_err, (cudaStream_t)stream);
  });
}

int he_launch_count(const he_ctx* c, uint64_t* out) {
  if (!c || !out) return fail(HE_EINVAL, "NULL argument");
  *out = c->launches.load();
  return HE_OK;
}

}  // extern "C"
