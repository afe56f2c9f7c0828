// Multi-right-hand-side M2L on the 5th-generation tensor cores (tcgen05, TF32 operands, FP32
// accumulators in tensor memory).
//
// For a target cluster t and its admissible sources s (Sec. 4.4), Y_t = sum_s S_ts X_s with S_ts the
// q^2 x q^2 complex coupling block and X_s the source expansions (q^2 x CR, CR = channels x R).  The
// complex product is formed from real ones: A = [Re S; Im S] (M = 128 rows: Re S in rows 0..q^2-1,
// Im S in rows 64..64+q^2-1) times B = [Re X | Im X] (N = 2 ns columns for a slice of ns complex
// columns), K = q^2 rounded up to 8; then Re Y = Re S Re X - Im S Im X and Im Y = Re S Im X + Im S Re X.
// FP32 accuracy from TF32 operands by the split v = hi + lo (hi = TF32(v), lo = TF32(v - hi)) and the
// three products hi hi + hi lo + lo hi.
//
// Accumulation: the tensor core sums into FP32 without rounding to nearest, and chaining the products
// of a whole interaction list into one accumulator lets those errors build up.  So each pair's
// product goes into a fresh tensor-memory buffer (two buffers, used alternately), which the CUDA cores
// add into FP32 registers (rounded to nearest) while the tensor core multiplies the next pair.
//
// Work split: one CTA per (target cluster, column group); a group is one or two slices of at most 64
// complex columns of one kernel type (hard: channel 0 is K, channels 1..6 are G), so each thread
// keeps at most 128 accumulators.  All 8 warps generate the coupling block (FP32, with the phase split
// of the FP32 path and the pair factor exp(i kappa |D|) folded in) straight into A.  The B operands
// (X_s split into TF32 hi / lo, already in operand layout) are packed once per matrix-vector product
// by k_m2l_tc_pack and streamed slice by slice by the bulk-copy engine into two buffers, the next
// slice loading while the current one multiplies.  One thread issues the MMAs and copies; mbarriers
// track their completion with waits bounded in time: a wait that runs out sets the status word, the
// CTA waits (bounded) for its copies and MMAs in flight, frees its tensor memory and returns without
// writing.
//
// Operand layout (no swizzle, K-major): core matrices of 8 rows x 16 bytes; element (row r, k) at byte
// ((r / 8) * KC + k / 4) * 128 + (r % 8) * 16 + (k % 4) * 4, KC = K / 4.  Descriptor: leading byte
// offset 128 (next core matrix along K), stride byte offset KC * 128 (next 8 rows).
#include <algorithm>
#include <cstdint>

#include "internal.h"
#include "k_m2l.cuh"
#include "kernels.h"

namespace igabem {

namespace {

constexpr int TC_THREADS = 256;
constexpr int TC_NS = 64;                                  // complex columns of a slice (N = 2 ns <= 128)
constexpr int TC_MAX_SLOTS = 8;
constexpr unsigned long long TC_WAIT_NS = 2000000000ull;   // bound of one mbarrier wait: 2 s

struct TCLevel {
  const int *far_ptr, *far_src;
  const float *nodes32;   // [7][n q^2]: x - c, n~, a
  const float *pc;        // pair constants [n_far][8]
  const uint8_t *bimg;    // packed B operands [n][hi / lo][2 CR rows x K]
  double2 *yhat;          // [n][q^2][CR]
  int n, first;
};

// slices: ns complex columns from column r0 (B rows 2 r0 .. 2 r0 + 2 ns: Re parts, then Im parts);
// groups: consecutive slices of one kernel type handled by one CTA
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

__device__ inline uint32_t tf32_bits(float v) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
  return r;
}

// byte offset of (r, k) in a K-major no-swizzle operand with KC core matrices along K
__device__ inline uint32_t op_off(int r, int k, int KC) {
  return (uint32_t)((((r >> 3) * KC + (k >> 2)) * 8 + (r & 7)) * 16 + (k & 3) * 4);
}

__device__ inline uint64_t smem_desc(uint32_t addr, int KC) {
  const uint64_t lbo = 128, sbo = (uint64_t)KC * 128;
  return (uint64_t)((addr >> 4) & 0x3FFF) | (((lbo >> 4) & 0x3FFF) << 16) | (((sbo >> 4) & 0x3FFF) << 32) |
         (1ull << 46);
}

__device__ inline void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
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

// wait for the completion of the phase with the given parity; false after TC_WAIT_NS
__device__ inline bool mbar_wait(uint32_t bar, uint32_t parity) {
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
      else if (t - t0 > TC_WAIT_NS) return false;
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

__global__ void __launch_bounds__(TC_THREADS, 1) k_m2l_tc(const TCArgs A) {
  extern __shared__ __align__(128) uint8_t smt[];
  __shared__ __align__(8) uint64_t bar_load[2], bar_free[2];
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  int li = 0;
  while (li + 1 < A.nlev && (int)blockIdx.x >= A.lev[li + 1].first) ++li;
  const TCLevel &L = A.lev[li];
  const int t = blockIdx.x - L.first;
  const int Q = A.Q, KH = A.KH, KC = KH >> 2, CR = A.CR;
  // this CTA's column group
  const int sl0 = A.sl.group_first[blockIdx.y], nsl = A.sl.group_n[blockIdx.y];
  const int type = A.sl.slot_type[sl0], gc0 = A.sl.slot_r0[sl0];
  int gcols = 0;
  for (int jj = 0; jj < nsl; ++jj) gcols += A.sl.slot_ns[sl0 + jj];
  const int W = 2 * gcols;  // tensor-memory columns of one pair buffer
  const uint32_t AB = 128u * KH * 4, BB = 2u * TC_NS * KH * 4;
  uint8_t *Ahi = smt, *Alo = smt + AB, *Bbuf = smt + 2 * AB;  // B buffer b: hi at 2 b BB, lo at (2 b + 1) BB
  float *tn = reinterpret_cast<float *>(smt + 2 * AB + 4 * BB);  // target nodes [64][9]
  float *sn = tn + 64 * 9;                                        // source nodes [64][8]
  const long NQ = (long)L.n * Q;
  const int k0 = L.far_ptr[t], npairs = L.far_ptr[t + 1] - k0;

  // A is zeroed once: the padding rows and columns are never written
  for (uint32_t i = tid; i < 2 * AB / 16; i += TC_THREADS) reinterpret_cast<uint4 *>(smt)[i] = make_uint4(0, 0, 0, 0);
  auto stage_nodes = [&](float *dst, int cl, int stride) {
    for (int a = tid; a < Q; a += TC_THREADS) {
      const long ia = (long)cl * Q + a;
      for (int c = 0; c < 7; ++c) dst[a * stride + c] = L.nodes32[c * NQ + ia];
    }
  };
  stage_nodes(tn, t, 9);
  if (npairs > 0) stage_nodes(sn, L.far_src[k0], 8);
  if (tid == 0) {
    for (int b = 0; b < 2; ++b) {
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
  const uint32_t idesc0 = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(128 >> 4) << 24);
  const uint32_t a_hi = smem_u32(Ahi), a_lo = smem_u32(Alo), b_base = smem_u32(Bbuf);

  const long total = (long)npairs * nsl;
  const size_t img_half = (size_t)2 * CR * KH * 4;
  // issuing thread state
  bool ok = true;
  long n_loaded = 0, n_mma = 0;
  auto issue_load = [&](long j) {
    const int p = (int)(j / nsl), sl = sl0 + (int)(j % nsl);
    const int s = L.far_src[k0 + p];
    const uint8_t *img = L.bimg + (size_t)s * 2 * img_half + (size_t)2 * A.sl.slot_r0[sl] * KH * 4;
    const uint32_t bytes = (uint32_t)2 * A.sl.slot_ns[sl] * KH * 4;
    const uint32_t b = (uint32_t)(j & 1), bar = smem_u32(&bar_load[b]);
    mbar_expect(bar, 2 * bytes);
    bulk_load(b_base + 2 * b * BB, img, bytes, bar);
    bulk_load(b_base + (2 * b + 1) * BB, img + img_half, bytes, bar);
    n_loaded = j + 1;
  };
  if (tid == 0 && total > 0) issue_load(0);

  // FP32 accumulators: TMEM lane 32 (warp % 4) + lane, columns [half W / 2, (half + 1) W / 2)
  float acc[8][16];
#pragma unroll
  for (int c = 0; c < 8; ++c)
#pragma unroll
    for (int i = 0; i < 16; ++i) acc[c][i] = 0.f;
  const int half = warp >> 2, nch = W / 32;
  auto drain = [&](int p) {  // adds pair p's buffer to the accumulators
    const uint32_t base = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)((p & 1) * A.wmax + half * (W / 2));
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      if (c < nch) {
        uint32_t v[16];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
            "[%16];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(base + 16 * c));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int i = 0; i < 16; ++i) acc[c][i] += __uint_as_float(v[i]);
      }
    }
  };

  const int ncq = (Q + 3) >> 2, ntile = ((Q + 7) >> 3) * ncq;
  const float kappa = A.kappa, eta = A.eta;
  int drained = 0;  // pairs added to the accumulators
  for (int p = 0; p < npairs; ++p) {
    const int kk = k0 + p;
    // A is rewritten: the MMAs of the previous pair must have read it
    if (tid == 0 && ok && n_mma > 0) ok = mbar_wait(smem_u32(&bar_free[(n_mma - 1) & 1]), (uint32_t)((n_mma - 1) >> 1) & 1);
    if (__syncthreads_or(tid == 0 && !ok)) break;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const float4 p0 = reinterpret_cast<const float4 *>(L.pc)[2 * kk];
    const float4 p1 = reinterpret_cast<const float4 *>(L.pc)[2 * kk + 1];
    const float D[3] = {p0.x, p0.y, p0.z};
    const float Dn = p0.w, D2 = p1.x;
    const C2<float> e0 = c2(p1.y, p1.z);
    for (int it = warp; it < ntile; it += TC_THREADS / 32) {
      const int a = (it / ncq) * 8 + (lane & 7), b = (it % ncq) * 4 + (lane >> 3);
      if (a >= Q || b >= Q) continue;
      const float *X = tn + a * 9, *Y = sn + b * 8;
      const C2<float> v = mul(e0, node_sample<float>(type, X, X + 3, X[6], Y, Y + 3, Y[6], D, Dn, D2, kappa, eta));
      const uint32_t rh = tf32_bits(v.x), ih = tf32_bits(v.y);
      const uint32_t o0 = op_off(a, b, KC), o1 = op_off(64 + a, b, KC);
      *reinterpret_cast<uint32_t *>(Ahi + o0) = rh;  // Re S
      *reinterpret_cast<uint32_t *>(Ahi + o1) = ih;  // Im S
      *reinterpret_cast<uint32_t *>(Alo + o0) = tf32_bits(v.x - __uint_as_float(rh));
      *reinterpret_cast<uint32_t *>(Alo + o1) = tf32_bits(v.y - __uint_as_float(ih));
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0 && ok) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      uint32_t off = (uint32_t)((p & 1) * A.wmax);
      for (int jj = 0; jj < nsl && ok; ++jj) {
        const long j = n_mma;
        const uint32_t b = (uint32_t)(j & 1);
        ok = mbar_wait(smem_u32(&bar_load[b]), (uint32_t)(j >> 1) & 1);
        if (!ok) break;
        const int ns = A.sl.slot_ns[sl0 + jj];
        const uint32_t idesc = idesc0 | ((uint32_t)((2 * ns) >> 3) << 17);
        const uint32_t bh = b_base + 2 * b * BB, bl = bh + BB;
        for (int ks = 0; ks < KH / 8; ++ks) {
          const uint32_t o = (uint32_t)ks * 256;
          mma_tf32(tmem + off, smem_desc(a_hi + o, KC), smem_desc(bh + o, KC), idesc, ks > 0 ? 1u : 0u);
          mma_tf32(tmem + off, smem_desc(a_hi + o, KC), smem_desc(bl + o, KC), idesc, 1u);
          mma_tf32(tmem + off, smem_desc(a_lo + o, KC), smem_desc(bh + o, KC), idesc, 1u);
        }
        mma_commit(smem_u32(&bar_free[b]));
        n_mma = j + 1;
        off += 2 * ns;
        // the next slice goes into the other buffer once the MMAs of item j - 1 have read it
        if (j + 1 < total) {
          if (j >= 1) ok = mbar_wait(smem_u32(&bar_free[(j - 1) & 1]), (uint32_t)((j - 1) >> 1) & 1);
          if (ok) issue_load(j + 1);
        }
      }
    }
    // while the tensor core multiplies pair p: add pair p - 1 and stage the next source's nodes
    if (p > 0) {
      drain(p - 1);
      drained = p;
    }
    if (p + 1 < npairs) stage_nodes(sn, L.far_src[kk + 1], 8);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  }
  // drain: every MMA and copy issued by this CTA completes before its memory is released
  if (tid == 0) {
    if (n_mma > 0) ok = mbar_wait(smem_u32(&bar_free[(n_mma - 1) & 1]), (uint32_t)((n_mma - 1) >> 1) & 1) && ok;
    for (long j = n_mma; j < n_loaded; ++j) ok = mbar_wait(smem_u32(&bar_load[j & 1]), (uint32_t)(j >> 1) & 1) && ok;
    if (!ok) atomicExch(A.status, 1);
  }
  const bool failed = __syncthreads_or(tid == 0 && !ok);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (!failed) {
    if (npairs > 0 && drained < npairs) drain(npairs - 1);
    // combine through shared memory (the B buffers are free): Y[a][c] for a < q^2, c < gcols
    double2 *Ys = reinterpret_cast<double2 *>(Bbuf);
    const int lrow = 32 * (warp & 3) + lane, a = lrow & 63;
    for (int pass = 0; pass < 2; ++pass) {
      // pass 0: Re S rows (lanes < 64) set Re Y += Re S Re X and Im Y += Re S Im X;
      // pass 1: Im S rows add Im Y += Im S Re X and Re Y -= Im S Im X
      if ((lrow >= 64) == (pass == 1) && a < Q) {
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          if (c < nch) {
#pragma unroll
            for (int i = 0; i < 16; ++i) {
              int col = half * (W / 2) + 16 * c + i, jj = 0, cc = 0;
              while (jj < nsl - 1 && col >= 2 * A.sl.slot_ns[sl0 + jj]) {
                col -= 2 * A.sl.slot_ns[sl0 + jj];
                cc += A.sl.slot_ns[sl0 + jj];
                ++jj;
              }
              const int ns = A.sl.slot_ns[sl0 + jj];
              const bool im_x = col >= ns;
              cc += im_x ? col - ns : col;
              double *y = reinterpret_cast<double *>(&Ys[a * 128 + cc]);
              const double v = acc[c][i];
              if (pass == 0) y[im_x ? 1 : 0] = v;
              else if (im_x) y[0] -= v;
              else y[1] += v;
            }
          }
        }
      }
      __syncthreads();
    }
    for (int i = tid; i < Q * gcols; i += TC_THREADS) {
      const int aa = i / gcols, c = i % gcols;
      L.yhat[((long)t * Q + aa) * CR + gc0 + c] = npairs > 0 ? Ys[aa * 128 + c] : make_double2(0.0, 0.0);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(A.tmem_cols) : "memory");
}

// B operands of one level: for cluster s, the 2 CR rows of the slices (slice rows 2 r0 .. 2 r0 + ns:
// Re xhat_s[b][r0 + i]; rows 2 r0 + ns + i: Im) by K = KH entries (k = b < q^2, zero beyond), split
// into TF32 hi and lo.  One block per (cluster, 8-row group): the group's 8 values per node are staged,
// then written in order.
__global__ void __launch_bounds__(256) k_m2l_tc_pack(const double2 *__restrict__ xhat, const TCSlices S, int Q,
                                                     int KH, int CR, uint8_t *__restrict__ bimg) {
  __shared__ float st[64 * 8];
  const int ng = (2 * CR) >> 3;
  const int s = blockIdx.x / ng, g = blockIdx.x % ng;
  int sl = 0;
  while (sl < S.nslot - 1 && 8 * g >= 2 * (S.slot_r0[sl] + S.slot_ns[sl])) ++sl;
  const int rel = 8 * g - 2 * S.slot_r0[sl], ns = S.slot_ns[sl];
  const bool im = rel >= ns;
  const int col0 = S.slot_r0[sl] + (im ? rel - ns : rel);
  for (int i = threadIdx.x; i < Q * 8; i += blockDim.x) {
    const int b = i >> 3, j = i & 7;
    const double2 v = xhat[((long)s * Q + b) * CR + col0 + j];
    st[i] = (float)(im ? v.y : v.x);
  }
  __syncthreads();
  const int KC = KH >> 2;
  uint32_t *hi = reinterpret_cast<uint32_t *>(bimg + (size_t)s * 2 * (2 * CR * KH * 4)) + (size_t)g * KC * 32;
  uint32_t *lo = hi + (size_t)2 * CR * KH;
  for (int i = threadIdx.x; i < KC * 32; i += blockDim.x) {
    const int kc = i >> 5, r8 = (i >> 2) & 7, k = kc * 4 + (i & 3);
    const float v = k < Q ? st[k * 8 + r8] : 0.f;
    const uint32_t h = tf32_bits(v);
    hi[i] = h;
    lo[i] = tf32_bits(v - __uint_as_float(h));
  }
}

int tc_kh(int Q) { return (Q + 7) / 8 * 8; }

size_t tc_smem_bytes(int KH) { return (size_t)2 * 128 * KH * 4 + (size_t)4 * 2 * TC_NS * KH * 4 + (64 * 9 + 64 * 8) * 4; }

// slices of at most 64 complex columns within one kernel type, grouped two by two
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
    for (int f = first; f < T.nslot; f += 2) {
      T.group_first[T.ngroup] = f;
      T.group_n[T.ngroup] = std::min(2, T.nslot - f);
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

bool m2l_tc_supported(const HostSetup &S, int R) {
  const int Q = S.q * S.q, CR = (S.hard ? 7 : 1) * R;
  if (Q > 64 || R % 16 != 0 || S.L - S.lmin + 1 > 16) return false;
  // slice count: hard R <= 64 gives 1 + 6, soft CR <= 512 gives 8
  if ((S.hard && R > TC_NS) || (!S.hard && CR > TC_MAX_SLOTS * TC_NS)) return false;
  return tc_smem_bytes(tc_kh(Q)) <= (size_t)max_optin_smem();
}

size_t m2l_tc_image_bytes(const HostSetup &S, int l, int R) {
  const int CR = (S.hard ? 7 : 1) * R;
  return (size_t)S.lev[l].n * 2 * (2 * CR) * tc_kh(S.q * S.q) * 4;
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
    for (int j = 0; j < A.sl.group_n[g]; ++j) w += 2 * A.sl.slot_ns[A.sl.group_first[g] + j];
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
    L.yhat = reinterpret_cast<double2 *>(d.yhat[l]);
    L.n = S.lev[l].n;
    L.first = nblocks;
    nblocks += S.lev[l].n;
    k_m2l_tc_pack<<<S.lev[l].n * (2 * A.CR / 8), 256, 0, st>>>(reinterpret_cast<const double2 *>(d.xhat[l]), A.sl,
                                                               A.Q, A.KH, A.CR, d.tc_bimg[l]);
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
