// Tensor-core Gram reduction C = A^T B with FP64-accurate products.
//
// Same result, partition and determinism as gram.cu (one synchronization point
// of the paper, Sec. 3), computed on the 5th-generation tensor cores instead of
// the GB300's narrow FP64 pipe.  The products are made exact by error-free
// splitting in the manner of Ozaki, Ogita, Oishi and Rump (Numer. Algorithms
// 59, 2012):
//
//   * every column i of A (and j of B) gets the exponent E_i with
//     max_r |a_ri| < 2^E_i (kept by the kernel that wrote the column, or found
//     by a column-max pass before the kernel);
//   * each entry becomes eight signed 8-bit digits relative to E_i, exact bf16
//     integers (tc_common.cuh);
//   * the 36 digit pairs t + u <= 7 run as bf16 tcgen05.mma with fp32
//     accumulation in tensor memory, one accumulator per level l = t + u,
//     exact over a 32-row block;
//   * after every block the eight level sums are read back (tcgen05.ld) and
//     added exactly into two int64 accumulators per output;
//   * at the end of its chunk a CTA writes 2^(E_i + E_j - 70) (hi 2^32 + lo)
//     as the FP64 chunk partial.
//
// The error of one product term is at most 2^-57.1 max|a_i| max|b_j| (dropped
// digit pairs and truncation); the integer sums are exact, so the chunk
// partial carries one FP64 rounding.  The partials are added in a fixed order
// (a function of the chunk count) by the reduction kernel of gram.cu.  (Fixed point relative to the column maximum
// loses log2(max|a_i| / |a_ri|) bits on small entries; 64 bits keep heavy-tailed
// columns, such as rows with lognormal norms, at FP64-level accuracy.)
//
// One CTA (512 threads) per (chunk, 128-column tile of A, 32-column tile of B),
// software-pipelined over 32-row blocks: cp.async stages block b+2 in shared
// memory while all threads split block b+1 into K-major bf16 digit tiles (one of
// two buffers) and the tensor cores run the MMAs of block b (issued by one
// thread, one per digit of A and 16-row step); then the warps read the level sums of block b back.  Every
// wait on the MMA barrier is bounded; on timeout the kernel records
// BCGS_ERR_TIMEOUT and returns after freeing its tensor memory.
#include <string.h>

#include "tc_common.cuh"

namespace bcgs {
namespace {
using namespace tc;

constexpr int kThreads = 512;
constexpr int kBlockRows = 32;          // rows (K) per MMA stage
constexpr int kChunks = kBlockRows / 8;  // 16-byte chunks of K per operand row in a digit tile
constexpr int kMTile = 128;              // A columns per CTA (MMA M)
constexpr int kATile = kMTile * kBlockRows * 2;  // bytes of one digit tile of A

struct TcCols {
  int32_t a_off[kMaxSegA + 1];
  int32_t b_off[kMaxSegB + 1];
  // per-column max |x| of each segment: kept by its writer or computed here
  const unsigned long long* a_amax[kMaxSegA];
  const unsigned long long* b_amax[kMaxSegB];
};

template <int MAXS>
__device__ __forceinline__ int find_seg(const int32_t* off, int nseg, int col) {
  int s = 0;
#pragma unroll
  for (int k = 1; k < MAXS; ++k)
    if (k < nseg && col >= off[k]) s = k;
  return s;
}

// Column max |x| of every column of one segment, kept as the bit pattern of
// |x|: for non-negative doubles unsigned order is value order, and Inf
// (0x7FF0...) and NaN (0x7FF8... and above) compare above every finite value,
// so a non-finite column shows as exponent field 0x7FF.
template <typename T>
__global__ void colmax_kernel(Seg S, int64_t m, unsigned long long* amax) {
  const int col = blockIdx.y;
  const int64_t off = (int64_t)col * S.ld;
  unsigned long long mx = 0ull;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < m;
       r += (int64_t)gridDim.x * blockDim.x)
    mx = umax64(mx, abs_bits64(ld_elem<T>(S.p, off + r)));
  warp_max_to(mx, amax + col);
}

__device__ __forceinline__ int cexp_of(unsigned long long b) { return (int)((b >> 52) & 0x7FF); }

template <typename T, int NBT>
__global__ void __launch_bounds__(kThreads, 1)
gram_tc_kernel(GramDesc d, TcCols cm, const unsigned long long* __restrict__ amax,
               double* __restrict__ partial, DevStatus* st) {
  static_assert(NBT == 16 || NBT == 32, "N tile");
  constexpr int kBTile = NBT * kBlockRows * 2;          // bytes of one digit tile of B
  constexpr int kStage = kDigits * (kATile + kBTile);  // one buffer of digit tiles
  constexpr int kCols = kMTile + NBT;                  // columns staged per block
  constexpr int kColBytes = kBlockRows * (int)sizeof(T) + 16;  // staged column, padded
  constexpr int kTmemCols = kDigits * NBT <= 128 ? 128 : (kDigits * NBT <= 256 ? 256 : 512);
  constexpr int kHalf = 8;                             // output columns per thread in the read-back
  constexpr int kGroups = NBT / kHalf;                 // column groups (warps w / 4 < kGroups read back)
  if (block_failed(st)) return;
  extern __shared__ uint8_t dyn[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base_s;
  __shared__ int s_cexp_a[kMTile];
  __shared__ int s_cexp_b[NBT];
  __shared__ const T* s_colptr[kCols];
  __shared__ int s_bad;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  uint8_t* digits = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(dyn) + 1023) & ~uintptr_t(1023));
  uint8_t* staging = digits + 2 * kStage;

  const int chunk = blockIdx.x;
  const int col0 = blockIdx.y * kMTile;       // first A column of this tile
  const int ncol_a = min(kMTile, d.na - col0);
  const int jb0 = blockIdx.z * NBT;           // first B column of this tile
  const int nb = min(NBT, d.nb - jb0);        // B columns of this tile
  const int ldp = d.nb;                       // row length of the partial layout
  const int64_t r_begin = (int64_t)chunk * d.chunk_rows;
  const int64_t r_end = min(r_begin + d.chunk_rows, d.m);

  if (tid == 0) s_bad = 0;
  __syncthreads();
  for (int i = tid; i < kMTile; i += kThreads) {
    int e = 0;
    const T* p = nullptr;
    if (i < ncol_a) {
      const int ca = col0 + i;
      const int sg = find_seg<kMaxSegA>(cm.a_off, d.nsa, ca);
      e = cexp_of(cm.a_amax[sg][ca - cm.a_off[sg]]);
      if (e == 0x7FF) s_bad = 1;
      p = reinterpret_cast<const T*>(d.a[sg].p) + (int64_t)(ca - cm.a_off[sg]) * d.a[sg].ld;
    }
    s_cexp_a[i] = e;
    s_colptr[i] = p;
  }
  for (int j = tid; j < NBT; j += kThreads) {
    int e = 0;
    const T* p = nullptr;
    if (j < nb) {
      const int cb = jb0 + j;
      const int sg = find_seg<kMaxSegB>(cm.b_off, d.nsb, cb);
      e = cexp_of(cm.b_amax[sg][cb - cm.b_off[sg]]);
      if (e == 0x7FF) s_bad = 1;
      p = reinterpret_cast<const T*>(d.b[sg].p) + (int64_t)(cb - cm.b_off[sg]) * d.b[sg].ld;
    }
    s_cexp_b[j] = e;
    s_colptr[kMTile + j] = p;
  }
  if (warp == 0) tmem_alloc<kTmemCols>(&tmem_base_s);
  if (tid == 0) mbar_init(&mbar);
  tc_before_sync();
  __syncthreads();
  tc_after_sync();
  const uint32_t tmem = tmem_base_s;
  const bool bad = s_bad != 0;
  if (bad && tid == 0) set_failure(st, BCGS_ERR_NONFINITE, d.block);
  const T* any_ptr = reinterpret_cast<const T*>(d.a[0].p);

  // global -> staging (column-major, one warp per 32 contiguous rows of a column)
  auto stage_copy = [&](int64_t r0) {
    for (int e = tid; e < kCols * kBlockRows; e += kThreads) {
      const int col = e / kBlockRows, r = e - col * kBlockRows;
      const T* p = s_colptr[col];
      const bool valid = p != nullptr && r0 + r < r_end;
      void* dst = staging + col * kColBytes + r * (int)sizeof(T);
      if constexpr (sizeof(T) == 8) cp_async8(dst, valid ? p + r0 + r : any_ptr, valid);
      else cp_async4(dst, valid ? p + r0 + r : any_ptr, valid);
    }
    cp_async_commit();
  };
  // staging -> digit tiles of buffer `buf`: task (column, 8-row group g); consecutive
  // threads take consecutive columns (conflict-free staging reads and tile writes)
  auto split_block = [&](int buf) {
    uint8_t* dA = digits + buf * kStage;
    uint8_t* dB = dA + kDigits * kATile;
    for (int e = tid; e < kCols * kChunks; e += kThreads) {
      const int g = e / kCols, col = e - g * kCols;
      const T* src = reinterpret_cast<const T*>(staging + col * kColBytes) + 8 * g;
      double v[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) v[k] = (double)src[k];
      if (col < kMTile) split8_interleave(v, s_cexp_a[col], dA, kATile, col, g, kChunks);
      else split8_interleave(v, s_cexp_b[col - kMTile], dB, kBTile, col - kMTile, g, kChunks);
    }
  };
  // One MMA per (digit t of A, 16-row K step): the B digit tiles are contiguous,
  // so [B_0 ... B_{8-t}] is a single K-major operand of (9-t) NBT rows whose
  // product with A_t lands, tile u, in the accumulator of level t + u (tensor
  // memory columns (t + u) NBT); pieces of at most 256 columns.
  auto issue_mma = [&](int buf) {
    const uint32_t a0 = smem_u32(digits + buf * kStage);
    const uint32_t b0 = a0 + kDigits * kATile;
    constexpr int kMaxLev = 256 / NBT;
#pragma unroll 1
    for (int t = 0; t < kDigits; ++t) {
      const int nlev = kDigits - t;
#pragma unroll 1
      for (int l0 = 0; l0 < nlev; l0 += kMaxLev) {
        const int nl = nlev - l0 < kMaxLev ? nlev - l0 : kMaxLev;
        const uint32_t id = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)((nl * NBT) >> 3) << 17) |
                            ((uint32_t)(kMTile >> 4) << 24);
        const uint32_t dcol = tmem + (uint32_t)((t + l0) * NBT);
#pragma unroll
        for (int kk = 0; kk < kBlockRows / 16; ++kk)
          mma_bf16(dcol, desc_interleave(a0 + t * kATile + kk * 256, 128, kChunks * 128),
                   desc_interleave(b0 + l0 * kBTile + kk * 256, 128, kChunks * 128), id,
                   (t == 0 && kk == 0) ? 0u : 1u);
      }
    }
    mma_commit(&mbar);
  };

  // read-back role: lane quadrant (warp % 4) -> A column, half (warp / 4) -> B columns
  const int my_i = 32 * (warp & 3) + lane;
  const int my_j0 = (warp >> 2) * kHalf;
  const bool reader = (warp >> 2) < kGroups;
  long long hi[kHalf], lo[kHalf];
#pragma unroll
  for (int j = 0; j < kHalf; ++j) hi[j] = lo[j] = 0;

  uint32_t phase = 0;
  bool timed_out = false;
  const int nblocks = bad ? 0 : (int)((r_end - r_begin + kBlockRows - 1) / kBlockRows);

  // Pipeline: block b's MMAs run while block b+1 is split; block b+2 is being
  // copied into the staging buffer meanwhile.
  if (nblocks > 0) {
    stage_copy(r_begin);
    cp_async_wait_all();
    __syncthreads();
    split_block(0);
    __syncthreads();
    if (nblocks > 1) stage_copy(r_begin + kBlockRows);
    fence_smem_to_async();
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    if (tid == 0) issue_mma(0);
  }
  for (int b = 0; b < nblocks; ++b) {
    const bool more = b + 1 < nblocks;
    if (more) {
      cp_async_wait_all();
      __syncthreads();
      split_block((b + 1) & 1);
      __syncthreads();
      if (b + 2 < nblocks) stage_copy(r_begin + (int64_t)(b + 2) * kBlockRows);
    }
    const bool ok = mbar_wait_bounded(&mbar, phase);
    phase ^= 1u;
    if (__syncthreads_or(!ok)) {
      timed_out = true;
      break;
    }
    tc_after_sync();
    // read back the exact level sums of block b and fold them
    const uint32_t lane_addr = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)my_j0;
    if (reader) {
#pragma unroll
    for (int g8 = 0; g8 < kHalf; g8 += 8) {
      int32_t L[8][kDigits];
#pragma unroll
      for (int l = 0; l < kDigits; ++l) {
        uint32_t r[8];
        tmem_ld8(lane_addr + (uint32_t)(l * NBT + g8), r);
#pragma unroll
        for (int j = 0; j < 8; ++j) L[j][l] = __float2int_rn(__uint_as_float(r[j]));
      }
#pragma unroll
      for (int j = 0; j < 8; ++j) fold_levels(L[j], hi[g8 + j], lo[g8 + j]);
    }
    }
    fence_smem_to_async();
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    if (more && tid == 0) issue_mma((b + 1) & 1);
  }
  cp_async_wait_all();

  // A CTA that saw a non-finite column or gave up on a wait writes NaN into its
  // partial slots: a caller without a status word (st == null) then gets NaN
  // from the reduction, never the sums some earlier call left in those slots.
  if (reader && my_i < ncol_a) {
    double* out = partial + (size_t)chunk * ((size_t)d.na * ldp) + (size_t)(col0 + my_i) * ldp + jb0;
    const int ea = s_cexp_a[my_i];
    const bool valid = !bad && !timed_out;
#pragma unroll
    for (int j = 0; j < kHalf; ++j) {
      const int jj = my_j0 + j;
      if (jj < nb) out[jj] = valid ? unfold(hi[j], lo[j], ea, s_cexp_b[jj]) : __longlong_as_double(0x7FF8000000000000LL);
    }
  }
  if (timed_out && tid == 0) set_failure(st, BCGS_ERR_TIMEOUT, d.block);
  tc_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc<kTmemCols>(tmem);
}


template <typename T>
cudaError_t launch_t(const GramDesc& d, double* partial, double* G, int ldg, unsigned long long* amax,
                     DevStatus* st, cudaStream_t stream) {
  TcCols cm;
  cm.a_off[0] = 0;
  for (int k = 0; k < kMaxSegA; ++k) cm.a_off[k + 1] = cm.a_off[k] + (k < d.nsa ? d.a[k].ncols : 0);
  cm.b_off[0] = 0;
  for (int k = 0; k < kMaxSegB; ++k) cm.b_off[k + 1] = cm.b_off[k] + (k < d.nsb ? d.b[k].ncols : 0);
  // column maxima: segments whose writer kept them are used as they are; the
  // others (at most once per distinct segment) are computed into `amax`
  {
    int64_t off = 0;
    int gx = (int)ceil_div(d.m, 256 * 64);
    if (gx > 16) gx = 16;
    if (gx < 1) gx = 1;
    const Seg* segs[kMaxSegA + kMaxSegB];
    const unsigned long long** dst[kMaxSegA + kMaxSegB];
    int ns = 0;
    for (int k = 0; k < d.nsa; ++k) { segs[ns] = &d.a[k]; dst[ns++] = &cm.a_amax[k]; }
    for (int k = 0; k < d.nsb; ++k) { segs[ns] = &d.b[k]; dst[ns++] = &cm.b_amax[k]; }
    for (int k = 0; k < ns; ++k) {
      const Seg& S = *segs[k];
      if (S.amax != nullptr) {
        *dst[k] = S.amax;
        continue;
      }
      const unsigned long long* same = nullptr;
      for (int q = 0; q < k; ++q)
        if (segs[q]->p == S.p && segs[q]->ld == S.ld && segs[q]->ncols >= S.ncols && segs[q]->amax == nullptr)
          same = *dst[q];
      if (same != nullptr) {
        *dst[k] = same;
        continue;
      }
      unsigned long long* out = amax + off;
      off += S.ncols;
      cudaError_t e = launch_zero_u64(out, S.ncols, stream);
      if (e != cudaSuccess) return e;
      colmax_kernel<T><<<dim3(gx, S.ncols), 256, 0, stream>>>(S, d.m, out);
      note_launch(1);
      *dst[k] = out;
    }
  }
  const int slot = prof_begin(stream);
  const int nbt = d.nb <= 16 ? 16 : 32;
  dim3 grid(d.nchunks, (unsigned)ceil_div(d.na, kMTile), (unsigned)ceil_div(d.nb, nbt));
#define BCGS_TC_CASE(NB)                                                                        \
  {                                                                                             \
    const size_t smem = 1024 + 2 * (size_t)kDigits * (kATile + NB * kBlockRows * 2) +           \
                        (size_t)(kMTile + NB) * (kBlockRows * sizeof(T) + 16);                  \
    cudaError_t e = ensure_dyn_smem(gram_tc_kernel<T, NB>, smem);                               \
    if (e != cudaSuccess) return e;                                                             \
    gram_tc_kernel<T, NB><<<grid, kThreads, smem, stream>>>(d, cm, amax, partial, st);           \
  }
  if (nbt == 16) BCGS_TC_CASE(16)
  else BCGS_TC_CASE(32)
#undef BCGS_TC_CASE
  prof_end(slot, kProfGramPartial, stream, 2.0 * (double)d.m * d.na * d.nb,
           (double)d.m * (d.na + d.nb) * sizeof(T) + (double)d.nchunks * d.na * d.nb * 8.0);
  note_launch(1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_gram_reduce(partial, d.nchunks, d.na, d.nb, G, ldg, st, stream);
}

}  // namespace

bool gram_tc_supported(const GramDesc& d) { return d.nb >= 1 && d.nb <= 64 && d.na >= 1; }

cudaError_t launch_gram_tc(const GramDesc& d, double* partial, double* G, int ldg,
                           unsigned long long* amax, DevStatus* st, cudaStream_t stream) {
  if (d.na <= 0 || d.nb <= 0) return cudaSuccess;
  const bool f32 = d.a[0].fp32 != 0;
  return f32 ? launch_t<float>(d, partial, G, ldg, amax, st, stream)
             : launch_t<double>(d, partial, G, ldg, amax, st, stream);
}

}  // namespace bcgs
