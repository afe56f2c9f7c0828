// Multi-right-hand-side M2L on the 5th-generation tensor cores (tcgen05, FP16 operands split into hi
// and lo parts, FP32 accumulators in tensor memory).
//
// For a target cluster t and its admissible sources s (Sec. 4.4), Y_t = sum_s S_ts X_s with S_ts the
// q^2 x q^2 complex coupling block and X_s the source expansions (q^2 x CR, CR = channels x R).  Each
// complex product is one real product in the 2 x 2 real form
//     [Re Y]   [Re S  -Im S] [Re X]
//     [Im Y] = [Im S   Re S] [Im X],
// so the MMA has M = 128 rows (Re rows 0..q^2-1, Im rows 64..64+q^2-1), K = 2 KH (Re X in k < q^2,
// Im X in KH <= k < KH + q^2, KH = q^2 rounded up to 8) and N = up to 64 right-hand-side columns per
// instruction.  FP32 accuracy from FP16 operands: every operand is first scaled by an exact power of two
// (per pair for S, from a bound on the kernel over the two clusters; per source cluster for X, from its
// largest entry) so that its entries lie well inside the FP16 range, then split v = hi + lo
// (hi = FP16(v), lo = FP16(v - hi)), and the three products hi hi + hi lo + lo hi are formed.
//
// Accumulation: the tensor core sums into FP32 without rounding to nearest, and chaining the products
// of a whole interaction list into one accumulator lets those errors build up.  So each pair's product
// goes into a fresh tensor-memory buffer (two buffers, used alternately), which the CUDA cores scale
// back (by the exact inverse powers of two) and add into FP32 registers, rounded to nearest.
//
// Work split: one CTA per (target cluster, column group); a group is up to four slices of at most 64
// columns of one kernel type (hard: channel 0 is K, channels 1..6 are G), so each thread keeps at most
// 128 accumulators.  Warps 1..7 generate the coupling block (FP32, with the phase split of the FP32
// path, the pair factor exp(i kappa |D|) and the pair's scale folded in) straight into A; A is
// double-buffered, so the block of pair p + 1 is generated, and pair p - 1 is added up, while the
// tensor core multiplies pair p.  The B operands (X_s scaled and split, already in operand layout) are
// packed once per matrix-vector product by k_m2l_tc_pack and streamed slice by slice by the bulk-copy
// engine into three buffers, two slices loading while one multiplies.  One thread of warp 0 issues the
// MMAs and copies; mbarriers track their completion with waits bounded in time: a wait that runs out
// sets the status word, the CTA waits (bounded) for its copies and MMAs in flight, frees its tensor
// memory and returns without writing.
//
// Operand layout (no swizzle, K-major): core matrices of 8 rows x 16 bytes (8 FP16); element (row r, k)
// at byte ((r / 8) * KC + k / 8) * 128 + (r % 8) * 16 + (k % 8) * 2, KC = K / 8.  Descriptor: leading
// byte offset 128 (next core matrix along K), stride byte offset KC * 128 (next 8 rows).
#include <cuda_fp16.h>

#include <algorithm>
#include <cstdint>

#include "internal.h"
#include "k_m2l.cuh"
#include "kernels.h"

namespace igabem {

namespace {

constexpr int TC_THREADS = 256;                            // 8 warps: warp 0 issues, 7 generate
constexpr int TC_NQW = TC_THREADS / 128;                   // warps per tensor-memory lane quadrant
constexpr int TC_MAXC = 16 / TC_NQW;                       // 16-column accumulator chunks per thread
constexpr int TC_NS = 64;                                  // columns of a slice (MMA N <= 64)
constexpr int TC_MAX_SLOTS = 8;
constexpr int TC_GROUP = 4;                                // slices per CTA (256 accumulator columns)
constexpr int TC_NBUF = 3;                                 // B buffers (two copies in flight)
constexpr unsigned long long TC_WAIT_NS = 2000000000ull;   // bound of one mbarrier wait: 2 s

struct TCLevel {
  const int *far_ptr, *far_src;
  const float *nodes32;   // [7][n q^2]: x - c, n~, a
  const float *pc;        // pair constants [n_far][8]; [7] = the pair's power-of-two scale
  const uint8_t *bimg;    // packed B operands [n][hi / lo][CR rows x K]
  const float *bscale;    // [n]: power-of-two scale of each cluster's packed operand
  double2 *yhat;          // [n][q^2][CR]
  int n, first;
};

// slices: ns columns from column r0 (B rows r0 .. r0 + ns); groups: consecutive slices of one kernel
// type handled by one CTA
struct TCSlices {
  int nslot, slot_r0[TC_MAX_SLOTS], slot_ns[TC_MAX_SLOTS], slot_type[TC_MAX_SLOTS];
  int ngroup, group_first[TC_MAX_SLOTS], group_n[TC_MAX_SLOTS];
};

struct TCArgs {
  TCLevel lev[16];
  TCSlices sl;
  int nlev, Q, KH, CR;
  int tmem_cols, wmax;    // tensor memory columns held; stride of the two pair buffers
  float kappa, eta;
  int *status;
};

__device__ inline uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// two FP32 values as FP16 hi parts (rounded to nearest) and FP16 lo parts (the rounded remainders),
// each pair packed in one 32-bit word (first value in the low half)
__device__ inline void split2(float v0, float v1, uint32_t &hi, uint32_t &lo) {
  const __half2 h = __floats2half2_rn(v0, v1);
  const float2 f = __half22float2(h);
  const __half2 l = __floats2half2_rn(v0 - f.x, v1 - f.y);
  hi = *reinterpret_cast<const uint32_t *>(&h);
  lo = *reinterpret_cast<const uint32_t *>(&l);
}

// byte offset of (r, k) (k even: a pair of FP16 values) in a K-major no-swizzle operand with KC core
// matrices (8 rows x 8 FP16) along K
__device__ inline uint32_t op_off(int r, int k, int KC) {
  return (uint32_t)((((r >> 3) * KC + (k >> 3)) * 8 + (r & 7)) * 16 + (k & 7) * 2);
}

__device__ inline uint64_t smem_desc(uint32_t addr, int KC) {
  const uint64_t lbo = 128, sbo = (uint64_t)KC * 128;
  return (uint64_t)((addr >> 4) & 0x3FFF) | (((lbo >> 4) & 0x3FFF) << 16) | (((sbo >> 4) & 0x3FFF) << 32) |
         (1ull << 46);
}

__device__ inline void mma_f16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ inline void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}

__device__ inline unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// wait for the completion of the phase with the given parity; false after limit_ns
__device__ inline bool mbar_wait(uint32_t bar, uint32_t parity, unsigned long long limit_ns = TC_WAIT_NS) {
  unsigned long long t0 = 0;
  for (unsigned it = 0;; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
    if ((it & 15) == 0) {
      const unsigned long long t = global_ns();
      if (t0 == 0) t0 = t;
      else if (t - t0 > limit_ns) return false;
    }
  }
}

__device__ inline void bulk_load(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

__device__ inline void mbar_expect(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// Constants of one pair for the generation of its coupling block.
struct TCPair {
  float D0, D1, D2, Dn, DD;  // D = c_t - c_s, |D|, |D|^2
  float phi0;                // kappa |D| reduced to (-pi, pi]
  float fs;                  // the pair's power-of-two scale / (4 pi)
};

// Kernel sample of type TYPE (0: soft K' - i eta V; 1: hard K; 2: hard G, as node_sample) times the
// pair factor exp(i kappa |D|) and the pair's scale.  Nodes in shared memory as three float4:
// [x - c, n~_x][n~_y, n~_z, a, 0][D.(x - c), D.n~, 0, 0] (the last one for sources only; for the
// target, Dx = D.(x - c) and Dnx = D.n~ are passed in).  The phase is kappa |D| + kappa (r - |D|)
// with r - |D| = (2 D.d + |d|^2) / (r + |D|), d the difference of the node offsets.
template <int TYPE>
__device__ inline float2 tc_sample(const TCPair &g, float kappa, float eta, const float4 &x0, const float4 &x1,
                                   float Dx, float Dnx, const float4 &y0, const float4 &y1, const float4 &y2) {
  const float d0 = x0.x - y0.x, d1 = x0.y - y0.y, d2 = x0.z - y0.z;
  const float dd = fmaf(d0, d0, fmaf(d1, d1, d2 * d2));
  const float num = fmaf(2.f, Dx - y2.x, dd);
  const float r2 = g.DD + num;
  const float ir = rsqrtf(r2), r = r2 * ir;
  float ph = fmaf(kappa, __fdividef(num, r + g.Dn), g.phi0);
  const float kq = rintf(ph * 0.15915494309189535f);
  ph = fmaf(-kq, 6.28318548202514648f, ph);
  ph = fmaf(-kq, -1.7484556e-07f, ph);
  float sph, cph;
  __sincosf(ph, &sph, &cph);
  const float f = ir * g.fs;
  if (TYPE == 2) return make_float2(cph * f, sph * f);
  const float kr = kappa * r, g2 = f * ir * ir;
  const float dGx = (-cph - sph * kr) * g2, dGy = (-sph + cph * kr) * g2;
  if (TYPE == 1) {  // -a_x ((x - y).n~_y) dG
    const float dn = y2.y + fmaf(d0, y0.w, fmaf(d1, y1.x, d2 * y1.y));
    const float w1 = -x1.z * dn;
    return make_float2(dGx * w1, dGy * w1);
  }
  // a_y ((x - y).n~_x) dG - i eta a_x a_y G
  const float dn = Dnx + fmaf(d0, x0.w, fmaf(d1, x1.x, d2 * x1.y));
  const float w1 = y1.z * dn, w2 = x1.z * y1.z * eta;
  return make_float2(fmaf(dGx, w1, sph * f * w2), fmaf(dGy, w1, -cph * f * w2));
}

// The coupling block of one pair into A (hi at Ahi, lo at Alo) by warps 1..7: 8 x 8 tiles (row
// a % 8 = lane % 8, column pair b, b + 1 with b % 8 = 2 (lane / 8)), two tiles per step for four
// independent samples in flight, stored as packed FP16 pairs (conflict-free within a core matrix).
template <int TYPE>
__device__ void tc_generate(const TCPair &g, float kappa, float eta, const float4 *__restrict__ tn4,
                            const float4 *__restrict__ sn4, uint8_t *__restrict__ Ahi, uint8_t *__restrict__ Alo,
                            int Q, int KH, int KC, int warp, int lane) {
  const int nb8 = (Q + 7) >> 3, ntile = nb8 * nb8, nw = TC_THREADS / 32 - 1;
  int it = warp - 1;
  int ag = it / nb8, bg = it % nb8;
  auto next = [&](int &ag_, int &bg_) {
    bg_ += nw;
    while (bg_ >= nb8) {
      bg_ -= nb8;
      ++ag_;
    }
  };
  while (it < ntile) {
    int ag2 = ag, bg2 = bg;
    next(ag2, bg2);
    const bool two = it + nw < ntile;
    float2 v[2][2];
    int aa[2], bb[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int a = (h ? ag2 : ag) * 8 + (lane & 7), b0 = (h ? bg2 : bg) * 8 + 2 * (lane >> 3);
      aa[h] = a;
      bb[h] = b0;
      v[h][0] = v[h][1] = make_float2(0.f, 0.f);
      if ((h == 0 || two) && a < Q && b0 < Q) {
        const float4 x0 = tn4[3 * a], x1 = tn4[3 * a + 1];
        const float Dx = fmaf(g.D0, x0.x, fmaf(g.D1, x0.y, g.D2 * x0.z));
        const float Dnx = TYPE == 0 ? fmaf(g.D0, x0.w, fmaf(g.D1, x1.x, g.D2 * x1.y)) : 0.f;
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int b = min(b0 + u, Q - 1);
          const float4 y0 = sn4[3 * b], y1 = sn4[3 * b + 1], y2 = sn4[3 * b + 2];
          const float2 w = tc_sample<TYPE>(g, kappa, eta, x0, x1, Dx, Dnx, y0, y1, y2);
          v[h][u] = b0 + u < Q ? w : make_float2(0.f, 0.f);
        }
      }
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int a = aa[h], b0 = bb[h];
      if ((h == 0 || two) && a < Q && b0 < Q) {
        uint32_t rh, rl, ih, il;
        split2(v[h][0].x, v[h][1].x, rh, rl);
        split2(v[h][0].y, v[h][1].y, ih, il);
        const uint32_t o00 = op_off(a, b0, KC), o01 = op_off(a, KH + b0, KC);
        const uint32_t o10 = op_off(64 + a, b0, KC), o11 = op_off(64 + a, KH + b0, KC);
        *reinterpret_cast<uint32_t *>(Ahi + o00) = rh;                // Re S
        *reinterpret_cast<uint32_t *>(Ahi + o01) = ih ^ 0x80008000u;  // -Im S
        *reinterpret_cast<uint32_t *>(Ahi + o10) = ih;                // Im S
        *reinterpret_cast<uint32_t *>(Ahi + o11) = rh;                // Re S
        *reinterpret_cast<uint32_t *>(Alo + o00) = rl;
        *reinterpret_cast<uint32_t *>(Alo + o01) = il ^ 0x80008000u;
        *reinterpret_cast<uint32_t *>(Alo + o10) = il;
        *reinterpret_cast<uint32_t *>(Alo + o11) = rl;
      }
    }
    it += 2 * nw;
    ag = ag2;
    bg = bg2;
    next(ag, bg);
  }
}

__global__ void __launch_bounds__(TC_THREADS, 1) k_m2l_tc(const TCArgs A) {
  extern __shared__ __align__(128) uint8_t smt[];
  __shared__ __align__(8) uint64_t bar_load[TC_NBUF], bar_free[TC_NBUF];
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  int li = 0;
  while (li + 1 < A.nlev && (int)blockIdx.x >= A.lev[li + 1].first) ++li;
  const TCLevel &L = A.lev[li];
  const int t = blockIdx.x - L.first;
  const int Q = A.Q, KH = A.KH, K = 2 * KH, KC = K >> 3, CR = A.CR;
  // this CTA's column group
  const int sl0 = A.sl.group_first[blockIdx.y], nsl = A.sl.group_n[blockIdx.y];
  const int type = A.sl.slot_type[sl0], gc0 = A.sl.slot_r0[sl0];
  int W = 0;  // columns of the group = tensor-memory columns of one pair buffer
  for (int jj = 0; jj < nsl; ++jj) W += A.sl.slot_ns[sl0 + jj];
  const uint32_t AB = 128u * K * 2, BB = (uint32_t)TC_NS * K * 2;
  uint8_t *Abuf = smt;            // A buffer u: hi at 2 u AB, lo at (2 u + 1) AB
  uint8_t *Bbuf = smt + 4 * AB;   // B buffer b: hi at 2 b BB, lo at (2 b + 1) BB
  float *tn = reinterpret_cast<float *>(smt + 4 * AB + 2 * TC_NBUF * BB);  // target nodes [64][12]
  float *snb = tn + 64 * 12;                                               // source nodes [2][64][12]
  const long NQ = (long)L.n * Q;
  const int k0 = L.far_ptr[t], npairs = L.far_ptr[t + 1] - k0;

  // both A buffers are zeroed once: the padding rows and columns are never written
  for (uint32_t i = tid; i < 4 * AB / 16; i += TC_THREADS) reinterpret_cast<uint4 *>(smt)[i] = make_uint4(0, 0, 0, 0);
  // nodes of cluster cl as [x - c, n~_x][n~_y, n~_z, a, 0][D.(x - c), D.n~, 0, 0] (D of pair kk) by the
  // threads lo .. lo + nt - 1
  auto stage_nodes = [&](float *dst, int cl, int kk, int lo, int nt) {
    float Dv[3] = {0.f, 0.f, 0.f};
    if (kk >= 0) {
      const float4 p0 = reinterpret_cast<const float4 *>(L.pc)[2 * kk];
      Dv[0] = p0.x;
      Dv[1] = p0.y;
      Dv[2] = p0.z;
    }
    for (int a = tid - lo; a < Q; a += nt) {
      const long ia = (long)cl * Q + a;
      float v[7];
      for (int c = 0; c < 7; ++c) v[c] = L.nodes32[c * NQ + ia];
      float4 *o = reinterpret_cast<float4 *>(dst + 12 * a);
      o[0] = make_float4(v[0], v[1], v[2], v[3]);
      o[1] = make_float4(v[4], v[5], v[6], 0.f);
      o[2] = make_float4(Dv[0] * v[0] + Dv[1] * v[1] + Dv[2] * v[2], Dv[0] * v[3] + Dv[1] * v[4] + Dv[2] * v[5], 0.f,
                         0.f);
    }
  };
  stage_nodes(tn, t, -1, 0, TC_THREADS);
  for (int p = 0; p < 2 && p < npairs; ++p) stage_nodes(snb + p * 768, L.far_src[k0 + p], k0 + p, 0, TC_THREADS);
  if (tid == 0) {
    for (int b = 0; b < TC_NBUF; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar_load[b])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar_free[b])));
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(A.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  const uint32_t idesc0 = (1u << 4) | ((uint32_t)(128 >> 4) << 24);  // FP32 accumulator, FP16 A and B, K-major
  const uint32_t a_base = smem_u32(Abuf), b_base = smem_u32(Bbuf);

  const long total = (long)npairs * nsl;
  const size_t img_half = (size_t)CR * K * 2;
  // issuing thread state
  bool ok = true;
  long n_loaded = 0, n_mma = 0;
  auto issue_load = [&](long j) {
    const int p = (int)(j / nsl), sl = sl0 + (int)(j % nsl);
    const int s = L.far_src[k0 + p];
    const uint8_t *img = L.bimg + (size_t)s * 2 * img_half + (size_t)A.sl.slot_r0[sl] * K * 2;
    const uint32_t bytes = (uint32_t)A.sl.slot_ns[sl] * K * 2;
    const uint32_t b = (uint32_t)(j % TC_NBUF), bar = smem_u32(&bar_load[b]);
    mbar_expect(bar, 2 * bytes);
    bulk_load(b_base + 2 * b * BB, img, bytes, bar);
    bulk_load(b_base + (2 * b + 1) * BB, img + img_half, bytes, bar);
    n_loaded = j + 1;
  };
  if (tid == 0)
    for (long j = 0; j < TC_NBUF - 1 && j < total; ++j) issue_load(j);

  // coupling block of pair p into A buffer p & 1 (source nodes in snb[p & 1]) by warps 1..7; warp 0
  // issues the MMAs
  const float kappa = A.kappa, eta = A.eta;
  auto generate = [&](int p) {
    if (warp > 0) {
      const int kk = k0 + p;
      const float4 p0 = reinterpret_cast<const float4 *>(L.pc)[2 * kk];
      const float4 p1 = reinterpret_cast<const float4 *>(L.pc)[2 * kk + 1];
      const TCPair g{p0.x, p0.y, p0.z, p0.w, p1.x, atan2f(p1.z, p1.y), p1.w * 0.0795774715459476679f};
      uint8_t *Ahi = Abuf + 2 * (p & 1) * AB, *Alo = Ahi + AB;
      const float4 *tn4 = reinterpret_cast<const float4 *>(tn);
      const float4 *sn4 = reinterpret_cast<const float4 *>(snb + (p & 1) * 768);
      if (type == 0)
        tc_generate<0>(g, kappa, eta, tn4, sn4, Ahi, Alo, Q, KH, KC, warp, lane);
      else if (type == 1)
        tc_generate<1>(g, kappa, eta, tn4, sn4, Ahi, Alo, Q, KH, KC, warp, lane);
      else
        tc_generate<2>(g, kappa, eta, tn4, sn4, Ahi, Alo, Q, KH, KC, warp, lane);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  };

  // FP32 accumulators: TMEM lane 32 (warp % 4) + lane; chunk c of the thread holds the group's
  // columns 16 (cq + NQW c) .. 16 (cq + NQW c) + 15 (cq = warp / 4, NQW warps per lane quadrant)
  float acc[TC_MAXC][16];
#pragma unroll
  for (int c = 0; c < TC_MAXC; ++c)
#pragma unroll
    for (int i = 0; i < 16; ++i) acc[c][i] = 0.f;
  const int cq = warp >> 2, nch = (W / 16 - cq + TC_NQW - 1) / TC_NQW;
  auto drain = [&](int p) {  // adds pair p's buffer, scaled back, to the accumulators
    const int kk = k0 + p;
    const float inv = 1.0f / (L.pc[8L * kk + 7] * L.bscale[L.far_src[kk]]);
    const uint32_t base = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)((p & 1) * A.wmax + 16 * cq);
#pragma unroll
    for (int c = 0; c < TC_MAXC; ++c) {
      if (c < nch) {
        uint32_t r[16];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
            "[%16];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(base + 16 * TC_NQW * c));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int i = 0; i < 16; ++i) acc[c][i] = fmaf(__uint_as_float(r[i]), inv, acc[c][i]);
      }
    }
  };

  if (npairs > 0) generate(0);
  // completion of item j (slice j % nsl of pair j / nsl): its buffer and the parity of its phase
  auto wait_free = [&](long j) { return mbar_wait(smem_u32(&bar_free[j % TC_NBUF]), (uint32_t)(j / TC_NBUF) & 1); };
  for (int p = 0; p < npairs; ++p) {
    // the MMAs of pair p - 1 have finished: its tensor-memory buffer is final and its A buffer (the one
    // pair p + 1 is generated into) is free
    if (tid == 0 && ok && p > 0) ok = wait_free((long)p * nsl - 1);
    if (__syncthreads_or(tid == 0 && !ok)) break;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (tid == 0) {
      const uint32_t ah = a_base + 2 * (p & 1) * AB, al = ah + AB;
      uint32_t off = (uint32_t)((p & 1) * A.wmax);
      for (int jj = 0; jj < nsl && ok; ++jj) {
        const long j = n_mma;
        const uint32_t b = (uint32_t)(j % TC_NBUF);
        ok = mbar_wait(smem_u32(&bar_load[b]), (uint32_t)(j / TC_NBUF) & 1);
        if (!ok) break;
        const int ns = A.sl.slot_ns[sl0 + jj];
        const uint32_t idesc = idesc0 | ((uint32_t)(ns >> 3) << 17);
        const uint32_t bh = b_base + 2 * b * BB, bl = bh + BB;
        for (int ks = 0; ks < K / 16; ++ks) {
          const uint32_t o = (uint32_t)ks * 256;
          mma_f16(tmem + off, smem_desc(ah + o, KC), smem_desc(bh + o, KC), idesc, ks > 0 ? 1u : 0u);
          mma_f16(tmem + off, smem_desc(ah + o, KC), smem_desc(bl + o, KC), idesc, 1u);
          mma_f16(tmem + off, smem_desc(al + o, KC), smem_desc(bh + o, KC), idesc, 1u);
        }
        mma_commit(smem_u32(&bar_free[b]));
        n_mma = j + 1;
        off += ns;
        // slice j + NBUF - 1 goes into the buffer of item j - 1 once its MMAs have read it
        const long jn = j + TC_NBUF - 1;
        if (jn < total && jn >= n_loaded) {
          if (j >= 1) ok = wait_free(j - 1);
          if (ok) issue_load(jn);
        }
      }
    }
    // while the tensor core multiplies pair p: add up pair p - 1, generate pair p + 1, stage the nodes
    // of pair p + 2 (into the buffer pair p used)
    if (p > 0) drain(p - 1);
    if (p + 1 < npairs) generate(p + 1);
    if (p + 2 < npairs && warp == 0) stage_nodes(snb + (p & 1) * 768, L.far_src[k0 + p + 2], k0 + p + 2, 0, 32);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  }
  // every MMA and copy issued by this CTA completes before its memory is released
  if (tid == 0) {
    if (n_mma > 0) ok = wait_free(n_mma - 1) && ok;
    for (long j = n_mma; j < n_loaded; ++j)
      ok = mbar_wait(smem_u32(&bar_load[j % TC_NBUF]), (uint32_t)(j / TC_NBUF) & 1) && ok;
    if (!ok) atomicExch(A.status, 1);
  }
  const bool failed = __syncthreads_or(tid == 0 && !ok);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (!failed) {
    if (npairs > 0) drain(npairs - 1);
    // through shared memory, 128 of the group's columns at a time: lanes 0..63 hold Re Y, lanes
    // 64..127 Im Y; Ys[a][c - w0] for a < q^2
    double2 *Ys = reinterpret_cast<double2 *>(smt);
    const int lrow = 32 * (warp & 3) + lane, a = lrow & 63;
    for (int w0 = 0; w0 < W; w0 += 128) {
      const int ww = min(128, W - w0);
      __syncthreads();
      if (a < Q) {
#pragma unroll
        for (int c = 0; c < TC_MAXC; ++c) {
          const int col = 16 * (cq + TC_NQW * c) - w0;
          if (c < nch && col >= 0 && col < 128)
#pragma unroll
            for (int i = 0; i < 16; ++i)
              reinterpret_cast<double *>(&Ys[a * 128 + col + i])[lrow < 64 ? 0 : 1] = (double)acc[c][i];
        }
      }
      __syncthreads();
      for (int i = tid; i < Q * ww; i += TC_THREADS) {
        const int aa = i / ww, c = i % ww;
        L.yhat[((long)t * Q + aa) * CR + gc0 + w0 + c] = Ys[aa * 128 + c];
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(A.tmem_cols) : "memory");
}

// Self-test of the bounded waits: one thread waits, with the routine the M2L uses, on an mbarrier that
// nothing arrives at; the wait must give up after limit_ns and the kernel reports it in status[0].
__global__ void k_wait_selftest(int *status, unsigned long long limit_ns) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    status[0] = mbar_wait(smem_u32(&bar), 0, limit_ns) ? 0 : 1;
  }
}

// B operands of one level, one block per cluster s: the cluster's scale 2^(12 - ceil(log2 max|X_s|))
// first (Re and Im parts), then the CR rows (columns of xhat_s) by K = 2 KH entries (Re xhat_s[b][r] at
// k = b, Im at k = KH + b, zero padding) scaled and split into FP16 hi and lo, written 8 rows at a time.
__global__ void __launch_bounds__(256) k_m2l_tc_pack(const double2 *__restrict__ xhat, int Q, int KH, int CR,
                                                     uint8_t *__restrict__ bimg, float *__restrict__ bscale) {
  __shared__ float2 st[64 * 8];
  __shared__ float wmax[8];
  const int s = blockIdx.x, K = 2 * KH, KC = K >> 3;
  const double2 *xs = xhat + (size_t)s * Q * CR;
  float m = 0.f;
  for (int i = threadIdx.x; i < Q * CR; i += blockDim.x) {
    const double2 v = xs[i];
    m = fmaxf(m, fmaxf(fabsf((float)v.x), fabsf((float)v.y)));
  }
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = m;
  __syncthreads();
  m = 0.f;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, wmax[w]);
  const float sigma = m > 0.f ? exp2f(12.f - ceilf(log2f(m))) : 1.f;
  if (threadIdx.x == 0) bscale[s] = sigma;
  uint32_t *hi = reinterpret_cast<uint32_t *>(bimg + (size_t)s * 2 * (CR * K * 2));
  uint32_t *lo = hi + (size_t)CR * K / 2;
  for (int g = 0; g < CR / 8; ++g) {
    __syncthreads();
    for (int i = threadIdx.x; i < Q * 8; i += blockDim.x) {
      const int b = i >> 3, j = i & 7;
      const double2 v = xs[(size_t)b * CR + 8 * g + j];
      st[i] = make_float2((float)v.x * sigma, (float)v.y * sigma);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < KC * 32; i += blockDim.x) {
      const int kc = i >> 5, r8 = (i >> 2) & 7, k = kc * 8 + 2 * (i & 3);
      float v[2];
      for (int u = 0; u < 2; ++u) {
        const int kk = k + u;
        v[u] = kk < Q ? st[kk * 8 + r8].x : (kk >= KH && kk < KH + Q ? st[(kk - KH) * 8 + r8].y : 0.f);
      }
      uint32_t h, l;
      split2(v[0], v[1], h, l);
      hi[(size_t)g * KC * 32 + i] = h;
      lo[(size_t)g * KC * 32 + i] = l;
    }
  }
}

// K = 2 KH must be a multiple of 16 (one MMA step); KH a multiple of 8 (one core matrix)
int tc_kh(int Q) { return (Q + 7) / 8 * 8; }

size_t tc_smem_bytes(int KH) {
  return (size_t)4 * 128 * (2 * KH) * 2 + (size_t)2 * TC_NBUF * TC_NS * (2 * KH) * 2 + (64 * 12 + 2 * 64 * 12) * 4;
}

// slices of at most 64 columns within one kernel type, grouped up to four at a time
TCSlices tc_slices(const HostSetup &S, int R) {
  TCSlices T{};
  const int CR = (S.hard ? 7 : 1) * R;
  auto add_type = [&](int r0, int r1, int type) {
    int first = T.nslot;
    for (int r = r0; r < r1; r += TC_NS) {
      T.slot_r0[T.nslot] = r;
      T.slot_ns[T.nslot] = std::min(TC_NS, r1 - r);
      T.slot_type[T.nslot] = type;
      ++T.nslot;
    }
    for (int f = first; f < T.nslot; f += TC_GROUP) {
      T.group_first[T.ngroup] = f;
      T.group_n[T.ngroup] = std::min(TC_GROUP, T.nslot - f);
      ++T.ngroup;
    }
  };
  if (S.hard) {
    add_type(0, R, 1);
    add_type(R, CR, 2);
  } else {
    add_type(0, CR, 0);
  }
  return T;
}

}  // namespace

void launch_wait_selftest(int *status, double limit_s, cudaStream_t st) {
  k_wait_selftest<<<1, 32, 0, st>>>(status, (unsigned long long)(limit_s * 1e9));
  IGA_CUDA(cudaGetLastError());
}

bool m2l_tc_supported(const HostSetup &S, int R) {
  const int Q = S.q * S.q, CR = (S.hard ? 7 : 1) * R;
  if (Q > 64 || R % 16 != 0 || S.L - S.lmin + 1 > 16) return false;
  for (int l = S.lmin; l <= S.L; ++l)
    if (S.lev[l].q != S.q) return false;  // one operand layout per launch: the same q on every level
  // slice count: hard R <= 64 gives 1 + 6, soft CR <= 512 gives 8
  if ((S.hard && R > TC_NS) || (!S.hard && CR > TC_MAX_SLOTS * TC_NS)) return false;
  return tc_smem_bytes(tc_kh(Q)) <= (size_t)max_optin_smem();
}

size_t m2l_tc_image_bytes(const HostSetup &S, int l, int R) {
  const int CR = (S.hard ? 7 : 1) * R;
  return (size_t)S.lev[l].n * 2 * CR * (2 * tc_kh(S.q * S.q)) * 2;
}

void launch_m2l_tc(const DeviceProblem &d, const HostSetup &S, const igabem_options &o, int R, cudaStream_t st) {
  TCArgs A;
  A.Q = S.q * S.q;
  A.KH = tc_kh(A.Q);
  A.CR = (S.hard ? 7 : 1) * R;
  A.kappa = (float)o.kappa;
  A.eta = (float)o.eta_cfie;
  A.status = d.status;
  A.sl = tc_slices(S, R);
  A.wmax = 0;
  for (int g = 0; g < A.sl.ngroup; ++g) {
    int w = 0;
    for (int j = 0; j < A.sl.group_n[g]; ++j) w += A.sl.slot_ns[A.sl.group_first[g] + j];
    A.wmax = std::max(A.wmax, w);
  }
  A.tmem_cols = 32;
  while (A.tmem_cols < 2 * A.wmax) A.tmem_cols *= 2;
  A.nlev = 0;
  int nblocks = 0;
  for (int l = S.lmin; l <= S.L; ++l) {
    TCLevel &L = A.lev[A.nlev++];
    L.far_ptr = d.far_ptr[l];
    L.far_src = d.far_src[l];
    L.nodes32 = d.nodes32[l];
    L.pc = d.pairc[l];
    L.bimg = d.tc_bimg[l];
    L.bscale = d.tc_bscale[l];
    L.yhat = reinterpret_cast<double2 *>(d.yhat[l]);
    L.n = S.lev[l].n;
    L.first = nblocks;
    nblocks += S.lev[l].n;
    k_m2l_tc_pack<<<S.lev[l].n, 256, 0, st>>>(reinterpret_cast<const double2 *>(d.xhat[l]), A.Q, A.KH, A.CR,
                                               d.tc_bimg[l], d.tc_bscale[l]);
    note_launch();
  }
  // at least 120 KB of shared memory per CTA: one CTA per SM, so tensor memory is never contended
  const size_t smem = std::max(tc_smem_bytes(A.KH), (size_t)120 * 1024);
  IGA_CUDA(set_max_dynamic_smem(k_m2l_tc, smem));
  dim3 grid(nblocks, A.sl.ngroup);
  k_m2l_tc<<<grid, TC_THREADS, smem, st>>>(A);
  note_launch();
  IGA_CUDA(cudaGetLastError());
}

}  // namespace igabem
