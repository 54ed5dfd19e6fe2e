// The synchronization Gram of a block step from the resident digit store:
//     G = A^T B,  A = store columns [0, na),  B = store columns [b0, b0 + nb)
// (Alg. 2: [Q_{1:k-1} U_k X_{k+1}]^T [U_k X_{k+1}]; the current U and X blocks
// sit in the store columns that Q fills next).  Nothing is split here: both
// operands are bulk copies of digit tiles, MN-major for the MMA (the 16-byte
// lines of the store run along the columns, the contraction along the rows).
//
// Both operands carry the store's seven leading digits (each value off by at
// most 2^-55 of its block column's maximum, so one product term by about
// 2^-53.9 of the product of the two maxima).  Per 128-row block b the digit
// products of one level are exact fp32 sums of 128 terms.  Block b's products carry the exponents E_bk (column k of A) and
// F_bj (column j of B); they are shifted onto the exponents Ec_k = max_b E_bk
// and Fc_j = max_b F_bj of the CTA's chunk of blocks (an exact right shift of
// the 128-bit fixed-point value, truncating at 2^-68 of the chunk maxima) and
// summed in int64 pairs.  The chunk partials go through the same ordered
// reduction as the other Gram kernels.
//
// One CTA per (chunk of blocks, 128-column tile of A): warp 8 issues the copies
// and the MMAs, warps 0..7 read the accumulators back; two accumulator sets in
// tensor memory let block b + 1 multiply while block b is read back.
#include <climits>

#include "tc_common.cuh"

namespace bcgs {

void gram_store_partition(int64_t m, int32_t* nchunks, int32_t* bpc) {
  const int64_t nblk = ceil_div(m, kStoreRows);
  const int64_t per = ceil_div(nblk, 152);  // one chunk per SM
  *bpc = (int32_t)per;
  *nchunks = (int32_t)ceil_div(nblk, per);
}

namespace {
using namespace tc;

constexpr int kWorkers = 256;
constexpr int kThreads = kWorkers + 32;
constexpr int kDigBytes = kStoreRows * kStoreCols * 2;  // one digit of a store tile: 32 KB

template <int NBT>
struct GSCfg {
  static constexpr int kAStages = NBT == 32 ? 3 : 4;
  static constexpr int kBDigit = NBT / 8 * 2048;  // one digit of B: NBT / 8 column groups
  // B's eight digit planes: seven from the store, the eighth stays zero (so the
  // first MMA of a block, digit 0 of A against planes 0..7, sets all eight levels)
  static constexpr int kBBuf = kDigits * kBDigit;
  static constexpr int kAcc = kDigits * NBT;
  static constexpr int kTmem = 2 * kAcc;
  static constexpr size_t kSmem = 1024 + (size_t)kAStages * kDigBytes + 2 * (size_t)kBBuf;
};

// v = hb 2^32 + lb as a 128-bit integer, shifted right by D (arithmetic), added
// to the pair (hi, lo) that stands for hi 2^32 + lo.
__device__ __forceinline__ void shift_add(long long hb, long long lb, int D, long long& hi, long long& lo) {
  const unsigned long long a = (unsigned long long)hb << 32;
  unsigned long long vl = a + (unsigned long long)lb;
  long long vh = (hb >> 32) + (lb >> 63) + (vl < a ? 1 : 0);
  if (D >= 64) {
    vl = (unsigned long long)(vh >> (D - 64 < 63 ? D - 64 : 63));
    vh >>= 63;
  } else if (D > 0) {
    vl = (vl >> D) | ((unsigned long long)vh << (64 - D));
    vh >>= D;
  }
  hi += (long long)(((unsigned long long)vh << 32) | (vl >> 32));
  lo += (long long)(vl & 0xFFFFFFFFull);
}

template <int NBT>
__global__ void __launch_bounds__(kThreads, 1) gram_store_kernel(GramStoreDesc d, double* partial,
                                                                 DevStatus* st) {
  using C = GSCfg<NBT>;
  constexpr int S = C::kAStages;
  constexpr int kHalf = NBT / 2;
  if (block_failed(st)) return;
  extern __shared__ uint8_t dyn[];
  __shared__ __align__(8) uint64_t fullA[S];
  __shared__ __align__(8) uint64_t doneA[S];
  __shared__ __align__(8) uint64_t fullB[2];
  __shared__ __align__(8) uint64_t accdone[2];
  __shared__ __align__(8) uint64_t accfree[2];
  __shared__ uint32_t tmem_base_s;
  __shared__ int s_Ec[kStoreCols];
  __shared__ int s_Fc[NBT];
  __shared__ int s_fail;

  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(dyn) + 1023) & ~uintptr_t(1023));
  uint8_t* Aring = base;
  uint8_t* Bbuf = Aring + S * kDigBytes;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // the column tiles of one chunk are adjacent in launch order, so they run at
  // the same time and the second read of the chunk's B digits hits L2
  const int G = blockIdx.x, ch = blockIdx.y;
  const QStore qs = d.qs;
  const int64_t b_first = (int64_t)ch * d.bpc;
  const int nbl = (int)min((int64_t)d.bpc, qs.nblk - b_first);
  const int ntot = nbl * kStoreDigits;  // A chunks: (block, digit)
  auto tile = [&](int64_t b, int g, int t) {
    return qs.dig + ((size_t)(b * qs.ngroups + g) * kStoreDigits + t) * kDigBytes;
  };

  if (tid == 0) {
    s_fail = 0;
    for (int i = 0; i < S; ++i) {
      mbar_init(&fullA[i]);
      mbar_init(&doneA[i]);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&fullB[i]);
      mbar_init(&accdone[i]);
      mbar_init_count(&accfree[i], kWorkers / 32);
    }
  }
  // B columns past the store stay zero
  for (int e = tid; e < 2 * C::kBBuf / 16; e += kThreads) reinterpret_cast<uint4*>(Bbuf)[e] = make_uint4(0, 0, 0, 0);
  // exponents shared by this chunk's blocks: the maxima over its blocks
  for (int col = tid; col < kStoreCols + NBT; col += kThreads) {
    const int gcol = col < kStoreCols ? kStoreCols * G + col : d.b0 + (col - kStoreCols);
    int mx = 0;
    if (gcol < qs.ld_exp) {
      const int32_t* e0 = qs.exps + b_first * qs.ld_exp + gcol;
      int bl = 0;
      for (; bl + 8 <= nbl; bl += 8) {
        int v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = e0[(int64_t)(bl + u) * qs.ld_exp];
#pragma unroll
        for (int u = 0; u < 8; ++u) mx = max(mx, v[u]);
      }
      for (; bl < nbl; ++bl) mx = max(mx, e0[(int64_t)bl * qs.ld_exp]);
    }
    if (col < kStoreCols) s_Ec[col] = mx;
    else s_Fc[col - kStoreCols] = mx;
  }
  if (warp == 0) tmem_alloc<C::kTmem>(&tmem_base_s);
  fence_smem_to_async();
  tc_before_sync();
  __syncthreads();
  tc_after_sync();
  const uint32_t tmem = tmem_base_s;

  if (warp == kWorkers / 32) {
    if (lane == 0) {
      // ---- copies and MMAs
      const int g_lo = d.b0 / 8;
      const int g_cnt = min(NBT / 8, qs.ngroups * 16 - g_lo);
      const int G1 = g_lo / 16, gs = g_lo % 16;
      const int n1 = min(g_cnt, 16 - gs), n2 = g_cnt - n1;
      // only the 8-column groups of the tile that hold columns < na (the rows of
      // the MMA beyond them read earlier, finite digits and are not written out)
      const int a_cols = min(kStoreCols, d.na - kStoreCols * G);
      const uint32_t a_bytes = (uint32_t)((a_cols + 7) / 8) * 2048u;
      auto issue_A = [&](int a) {
        const int slot = a % S;
        mbar_arrive_expect_tx(&fullA[slot], a_bytes);
        bulk_g2s(Aring + slot * kDigBytes, tile(b_first + a / kStoreDigits, G, a % kStoreDigits), a_bytes,
                 &fullA[slot]);
      };
      auto issue_B = [&](int bl) {
        const int p = bl & 1;
        mbar_arrive_expect_tx(&fullB[p], (uint32_t)(kStoreDigits * g_cnt * 2048));
        const int64_t b = b_first + bl;
        for (int u = 0; u < kStoreDigits; ++u) {
          uint8_t* dst = Bbuf + p * C::kBBuf + u * C::kBDigit;
          if (n1 > 0) bulk_g2s(dst, tile(b, G1, u) + gs * 2048, n1 * 2048, &fullB[p]);
          if (n2 > 0) bulk_g2s(dst + n1 * 2048, tile(b, G1 + 1, u), n2 * 2048, &fullB[p]);
        }
      };
      bool ok = true;
      int issuedA = 0, issuedB = 0, gotA = 0, gotB = 0;
      for (; issuedB < 2 && issuedB < nbl; ++issuedB) issue_B(issuedB);
      for (; issuedA < S && issuedA < ntot; ++issuedA) issue_A(issuedA);
      // Event loop: A slots and B buffers are refilled as soon as the MMAs that
      // read them are done, and a chunk's MMAs go out as soon as its operands are
      // ready, so every copy slot stays in flight while the tensor core waits.
      // No progress for kWaitCycles ends the loop with a failure.
      int a = 0, need = 0;  // chunk a = (block a / 7, digit a % 7); need: 0 = B, 1 = accumulator, 2 = A
      long long idle0 = clock64();
      while (a < ntot) {
        bool progress = false;
        const int xa = issuedA - S;  // the chunk that last used the slot of chunk issuedA
        if (issuedA < ntot && xa < a && mbar_test(&doneA[xa % S], (xa / S) & 1)) {
          issue_A(issuedA);
          ++issuedA;
          progress = true;
        }
        // B of block issuedB into the buffer of block issuedB - 2 once all its MMAs are done
        const int xb = issuedB - 2;
        if (issuedB < nbl && (xb + 1) * kStoreDigits <= a && mbar_test(&accdone[xb & 1], (xb >> 1) & 1)) {
          issue_B(issuedB);
          ++issuedB;
          progress = true;
        }
        const int bl = a / kStoreDigits, t = a % kStoreDigits, p = bl & 1, slot = a % S;
        if (need == 0) {
          if (t != 0) {
            need = 1;
          } else if (mbar_test(&fullB[p], (bl >> 1) & 1)) {
            gotB = bl + 1;
            need = 1;
          }
        }
        if (need == 1 && (t != 0 || bl < 2 || mbar_test(&accfree[p], ((bl >> 1) - 1) & 1))) need = 2;
        if (need == 2 && mbar_test(&fullA[slot], (a / S) & 1)) {
          gotA = a + 1;
          tc_after_sync();
          const uint32_t acc = tmem + (uint32_t)(p * C::kAcc + t * NBT);
          const uint32_t a0 = smem_u32(Aring + slot * kDigBytes);
          const uint32_t b0 = smem_u32(Bbuf + p * C::kBBuf);
          // both operands MN-major: (LBO, SBO) = (K-direction, MN-direction) core strides
          // digit t of A (t < 7: the store keeps seven) times B's planes u <= 7 - t
          // (plane 7 is zero): levels t .. 7
          const uint32_t id = idesc_f16(kStoreRows, (kDigits - t) * NBT) | (1u << 15) | (1u << 16);
#pragma unroll
          for (int ks = 0; ks < kStoreRows / 16; ++ks)
            mma_bf16(acc, desc_interleave(a0 + ks * 256, 128, 2048), desc_interleave(b0 + ks * 256, 128, 2048), id,
                     (t == 0 && ks == 0) ? 0u : 1u);
          mma_commit(&doneA[slot]);
          if (t == kStoreDigits - 1) mma_commit(&accdone[p]);
          ++a;
          need = 0;
          progress = true;
        }
        if (progress) {
          idle0 = clock64();
        } else if (clock64() - idle0 > kWaitCycles) {
          ok = false;
          break;
        }
      }
      if (!ok) {
        s_fail = 1;
        // copies still in flight land before the CTA's shared memory goes away
        for (int x = gotA; x < issuedA; ++x) mbar_wait_bounded(&fullA[x % S], (x / S) & 1);
        for (int x = gotB; x < issuedB; ++x) mbar_wait_bounded(&fullB[x & 1], (x >> 1) & 1);
      }
    }
  }

  // ---- read-back (warps 0..7): lane = column k of the A tile, kHalf columns j of B
  const int my_k = 32 * (warp & 3) + lane;
  const int j0 = (warp >> 2) * kHalf;
  const int gk = kStoreCols * G + my_k;
  long long hi[kHalf], lo[kHalf];
#pragma unroll
  for (int j = 0; j < kHalf; ++j) hi[j] = lo[j] = 0;
  bool wok = true;
  if (warp < kWorkers / 32) {
    const int Ec = s_Ec[my_k];
    int Fc[kHalf];
#pragma unroll
    for (int j = 0; j < kHalf; ++j) Fc[j] = s_Fc[j0 + j];
    auto load_e = [&](int bl, int& ea, int (&eb)[kHalf]) {
      const int32_t* row = qs.exps + (b_first + bl) * qs.ld_exp;
      ea = gk < qs.ld_exp ? row[gk] : 0;
#pragma unroll
      for (int j = 0; j < kHalf; ++j) {
        const int col = d.b0 + j0 + j;
        eb[j] = col < qs.ld_exp ? row[col] : 0;
      }
    };
    int ea, eb[kHalf];
    load_e(0, ea, eb);
    for (int bl = 0; bl < nbl; ++bl) {
      const int p = bl & 1;
      int ea_n = 0, eb_n[kHalf];
#pragma unroll
      for (int j = 0; j < kHalf; ++j) eb_n[j] = 0;
      if (bl + 1 < nbl) load_e(bl + 1, ea_n, eb_n);
      wok = __all_sync(0xffffffffu, mbar_wait_bounded(&accdone[p], (bl >> 1) & 1));
      if (!wok) break;
      tc_after_sync();
      const uint32_t addr = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(p * C::kAcc + j0);
#pragma unroll
      for (int g8 = 0; g8 < kHalf; g8 += 8) {
        long long hb[8], lb[8];
#pragma unroll
        for (int half = 0; half < 2; ++half) {
          uint32_t r[4][8];
#pragma unroll
          for (int l = 0; l < 4; ++l) tmem_ld8_nowait(addr + (uint32_t)((4 * half + l) * NBT + g8), r[l]);
          tmem_wait_ld();
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int32_t L0 = __float2int_rn(__uint_as_float(r[0][j]));
            const int32_t L1 = __float2int_rn(__uint_as_float(r[1][j]));
            const int32_t L2 = __float2int_rn(__uint_as_float(r[2][j]));
            const int32_t L3 = __float2int_rn(__uint_as_float(r[3][j]));
            if (half == 0)
              hb[j] = ((long long)((L0 << 8) + L1) << 16) + (long long)((L2 << 8) + L3);
            else
              lb[j] = ((long long)L0 << 24) + ((long long)L1 << 16) + ((long long)L2 << 8) + (long long)L3;
          }
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int e2 = eb[g8 + j];
          if (ea != 0 && e2 != 0) {
            int D = (Ec - ea) + (Fc[g8 + j] - e2);
            D = D < 0 ? 0 : (D > 127 ? 127 : D);
            shift_add(hb[j], lb[j], D, hi[g8 + j], lo[g8 + j]);
          }
        }
      }
      tc_before_sync();
      __syncwarp();
      if (lane == 0) mbar_arrive(&accfree[p]);
      ea = ea_n;
#pragma unroll
      for (int j = 0; j < kHalf; ++j) eb[j] = eb_n[j];
    }
  }
  tc_before_sync();
  __syncthreads();
  const bool fail = s_fail != 0 || !__syncthreads_and(wok);
  if (warp < kWorkers / 32 && !fail && gk < d.na) {
    const int Ec = s_Ec[my_k];
    const size_t nout = (size_t)d.na * d.nb;
    double* out = partial + (size_t)ch * nout + (size_t)gk * d.nb;
#pragma unroll
    for (int j = 0; j < kHalf; ++j) {
      const int jj = j0 + j;
      const int Fc = s_Fc[jj];
      if (jj < d.nb) out[jj] = (Ec == 0 || Fc == 0) ? 0.0 : fixed_to_double(hi[j], lo[j], Ec + Fc - 1022);
    }
  }
  if (fail && tid == 0) set_failure(st, BCGS_ERR_TIMEOUT, d.block);
  if (warp == 0) tmem_dealloc<C::kTmem>(tmem);
}

template <int NBT>
cudaError_t launch_gs(const GramStoreDesc& d, double* partial, DevStatus* st, cudaStream_t stream) {
  const size_t smem = GSCfg<NBT>::kSmem;
  cudaError_t e = ensure_dyn_smem(gram_store_kernel<NBT>, smem);
  if (e != cudaSuccess) return e;
  const dim3 grid((unsigned)ceil_div(d.na, kStoreCols), (unsigned)d.nchunks);
  gram_store_kernel<NBT><<<grid, kThreads, smem, stream>>>(d, partial, st);
  return cudaSuccess;
}

// The timeout path without a fault: the barrier expects one arrival that never
// comes, so the bounded wait gives up after `cycles` and the kernel records
// BCGS_ERR_TIMEOUT, as every bounded wait of the library does.
__global__ void wait_selftest_kernel(DevStatus* st, long long cycles) {
  __shared__ __align__(8) uint64_t mbar;
  if (threadIdx.x == 0) mbar_init(&mbar);
  __syncthreads();
  if (threadIdx.x == 0 && !mbar_wait_limit(&mbar, 0, cycles)) set_failure(st, BCGS_ERR_TIMEOUT, 0);
}

}  // namespace

cudaError_t launch_wait_selftest(DevStatus* st, long long cycles, cudaStream_t stream) {
  wait_selftest_kernel<<<1, 32, 0, stream>>>(st, cycles);
  note_launch(1);
  return cudaGetLastError();
}

bool gram_store_supported(int32_t na, int32_t b0, int32_t nb) {
  return na >= 1 && nb >= 1 && nb <= 32 && b0 >= 0 && b0 % 8 == 0;
}

cudaError_t launch_gram_store(const GramStoreDesc& d, double* partial, double* G, int32_t ldg, DevStatus* st,
                              cudaStream_t stream) {
  if (!gram_store_supported(d.na, d.b0, d.nb) || d.b0 + d.nb > d.qs.ld_exp || d.na > d.qs.ld_exp)
    return cudaErrorInvalidValue;
  if (d.m == 0) return cudaSuccess;
  const int slot = prof_begin(stream);
  const cudaError_t e = d.nb <= 16 ? launch_gs<16>(d, partial, st, stream) : launch_gs<32>(d, partial, st, stream);
  if (e != cudaSuccess) return e;
  prof_end(slot, kProfGramPartial, stream, 2.0 * (double)d.m * d.na * d.nb, 8.0 * (double)d.m * (d.na + d.nb));
  note_launch(1);
  const cudaError_t e2 = cudaGetLastError();
  if (e2 != cudaSuccess) return e2;
  return launch_gram_reduce(partial, d.nchunks, d.na, d.nb, G, ldg, st, stream);
}

}  // namespace bcgs
