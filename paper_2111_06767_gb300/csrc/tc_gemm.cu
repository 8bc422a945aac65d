// Subdomain-inverse GEMM on the 5th-generation tensor cores (tcgen05, TF32 inputs, FP32 accumulate).
//
// du_S = A_S^-1 r_S for all subdomains of a class (Sec. III.E, explicit-inverse solver) is the one
// dense contraction of the method: Y[:, cols] = Inv_c (ld x ld, row-major) * X[:, cols] with every
// subdomain column of X contiguous. Both operands are K-major, so each CTA computes a 128 x BN
// output tile (BN = 64, or 128 / 256 so that a class of at most that many subdomains reads each
// 128-row slab of its inverse once): TMA streams 128 x 32 tiles of Inv_c and BN x 32 tiles of X
// (128-byte swizzle) into a 3- or 4-stage shared-memory ring, one elected thread issues
// tcgen05.mma (M = 128, N = BN, K = 8 per instruction) accumulating in tensor memory, and the four
// warps read the accumulator back with tcgen05.ld and store it column-contiguously. Only the K
// chunks that meet a slot of the subdomain present in the class are streamed (the slots of missing
// neighbours have zero coupling), and tiles whose rows lie only in such slots write zeros without
// a K loop. When the tiles alone cannot fill the GPU, the K range is split across a cluster of 2,
// 4 or 8 CTAs and the partial tiles are summed through distributed shared memory in a fixed order.
// Every wait is bounded: on timeout the CTA raises an error flag, drains and frees its tensor
// memory.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>
#include <set>

#include "internal.h"
#include "pdl.cuh"

namespace dg {

namespace {

constexpr int BM = 128, BK = 32;
constexpr int A_BYTES = BM * BK * 4;  // 16 KiB
constexpr int SLACK = 8 * 1024;       // spare shared memory after the ring
constexpr uint32_t WAIT_LIMIT = 1u << 20;  // polls before a wait gives up (far above any real wait)

// Shape constants of the tile width BN (64, 128 or 256).
template <int BN>
struct TcShape {
  static constexpr int STAGES = BN == 128 ? 3 : 4;  // TMA ring depth (two CTAs per SM up to BN = 128)
  static constexpr int B_BYTES = BN * BK * 4;  // 8, 16 or 32 KiB
  static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
  static constexpr int TMEM_COLS = BN < 128 ? 128 : BN;  // >= BN, a power of two
  static constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + SLACK + 1024 + 256;
  static constexpr int PER_SM = BN <= 128 ? 2 : 1;     // co-resident CTAs per SM
  static constexpr int SLOTS = PER_SM * 152;
  // instruction descriptor: F32 accumulate, TF32 A and B, both K-major, N = BN, M = BM
  static constexpr uint32_t IDESC =
      (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
  static_assert(BN % 16 == 0 && BN >= 16 && BN <= 256, "tcgen05.mma with M = 128 takes N = 16..256");
  static_assert(BM * BN * 4 <= STAGES * STAGE_BYTES, "split-K partial tile must fit in the idle ring");
  static_assert(SMEM_BYTES <= 227 * 1024, "shared memory per CTA");
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred P1;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, P1;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait on an mbarrier phase; false (and the error flag set) if it never completes.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int* err) {
  for (uint32_t i = 0; i < WAIT_LIMIT; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  atomicExch(err, 1);
  return false;
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int c0, int c1,
                                            int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(dst),
      "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int c0, int c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
          "r"(dst),
      "l"(map), "r"(c0), "r"(c1), "r"(bar)
      : "memory");
}

// Shared-memory matrix descriptor for a K-major operand in the 128-byte swizzle layout written
// by TMA: rows of 128 bytes, 8-row swizzle atoms 1024 bytes apart.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);  // start address
  d |= (uint64_t)(16 >> 4) << 16;           // leading-dimension byte offset (single atom along K)
  d |= (uint64_t)(1024 >> 4) << 32;         // stride-dimension byte offset between 8-row groups
  d |= (uint64_t)1 << 46;                   // descriptor version
  d |= (uint64_t)2 << 61;                   // 128-byte swizzle
  return d;
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred P1;\n\t"
      "setp.ne.b32 P1, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, P1;\n\t}" ::"r"(tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, "
      "[%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Address of the same shared-memory location in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t map_peer(uint32_t local_addr, uint32_t rank) {
  uint32_t remote;
  asm("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(local_addr), "r"(rank));
  return remote;
}

// Plain (reorderable) load from a peer's shared memory; callers order it after the writes with a
// cluster barrier, which carries the memory clobber.
__device__ __forceinline__ float ld_cluster(uint32_t addr) {
  float v;
  asm("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(addr));
  return v;
}

// SPLIT > 1: the K range of a tile is split across the SPLIT CTAs of a thread-block cluster; each
// keeps its partial 128 x BN tile in shared memory and, after a cluster barrier, every CTA sums a
// 1/SPLIT of the tile's columns over all partials through distributed shared memory in
// rank order, so the result does not depend on timing.
template <int SPLIT, int BN>
__global__ void __launch_bounds__(128, TcShape<BN>::PER_SM)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                   float* __restrict__ Y, int ld, const int4* __restrict__ tiles, const int* __restrict__ kchunks,
                   int* __restrict__ err, float alpha) {
  using SH = TcShape<BN>;
  constexpr int STAGES = SH::STAGES;
  constexpr int B_BYTES = SH::B_BYTES, STAGE_BYTES = SH::STAGE_BYTES, TMEM_COLS = SH::TMEM_COLS;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* sA = smem;
  unsigned char* sB = smem + STAGES * A_BYTES;
  uint64_t* bars = (uint64_t*)(smem + STAGES * STAGE_BYTES + SLACK);  // full[STAGES], empty[STAGES], acc
  uint32_t* tmem_slot = (uint32_t*)(bars + 2 * STAGES + 1);
  int* s_issued = (int*)(tmem_slot + 1);    // TMA chunks issued by the producer
  int* s_consumed = (int*)(tmem_slot + 2);  // chunks the MMA thread saw arrive

  const int split = SPLIT > 1 ? (int)cluster_rank() : 0;
  const int4 tile = tiles[blockIdx.x / SPLIT];
  const int cls = tile.x & 0xFFFF, row0 = tile.y, col0 = tile.z, ncol = min(tile.w, BN);
  const bool zero = (tile.x >> 30) & 1;  // rows only in the slots of missing neighbours: zeros
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // the K chunks of this class that meet a present slot (the rest of the inverse's row is zero)
  const int* kl = kchunks + (size_t)cls * (ld / BK + 1);
  const int nk_all = zero ? 0 : kl[0];
  const int kc0 = split * nk_all / SPLIT, kc1 = (split + 1) * nk_all / SPLIT;
  const int nk = kc1 - kc0;
  ++kl;
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + STAGES), accb = smem_u32(bars + 2 * STAGES);

  if (threadIdx.x == 0) {
    *s_issued = 0;
    *s_consumed = 0;
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    mbar_init(accb, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  // set-up above overlaps the previous kernel; X (and Y) belong to the stream order from here on
  pdl_launch_dependents();
  pdl_wait();

  if (warp == 0 && lane == 0) {
    // producer: TMA loads into the ring
    for (int kc = 0; kc < nk; ++kc) {
      const int s = kc % STAGES;
      if (kc >= STAGES && !mbar_wait(empty0 + 8 * s, ((kc / STAGES) & 1) ^ 1, err)) break;
      mbar_expect_tx(full0 + 8 * s, STAGE_BYTES);
      const int k0 = kl[kc0 + kc] * BK;
      tma_load_3d(smem_u32(sA + s * A_BYTES), &mapA, full0 + 8 * s, k0, row0, cls);
      tma_load_2d(smem_u32(sB + s * B_BYTES), &mapB, full0 + 8 * s, k0, col0);
      *s_issued = kc + 1;
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer: 4 instructions of K = 8 per 32-wide K chunk
    for (int kc = 0; kc < nk; ++kc) {
      const int s = kc % STAGES;
      if (!mbar_wait(full0 + 8 * s, (kc / STAGES) & 1, err)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a0 = smem_u32(sA + s * A_BYTES), b0 = smem_u32(sB + s * B_BYTES);
#pragma unroll
      for (int kk = 0; kk < BK / 8; ++kk)
        mma_tf32(tmem, smem_desc(a0 + 32 * kk), smem_desc(b0 + 32 * kk), SH::IDESC, (kc | kk) != 0);
      mma_commit(empty0 + 8 * s);  // frees the stage once these MMAs have read it
      *s_consumed = kc + 1;
    }
    mma_commit(accb);
  }
  __syncwarp();

  // epilogue: warp w owns accumulator lanes (rows) 32 w .. 32 w + 31
  const bool ok = __all_sync(0xffffffffu, mbar_wait(accb, 0, err));
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const int r_local = warp * 32 + lane;
  const int row = row0 + r_local;
  const bool acc = nk > 0;  // the accumulator holds a product (else this CTA's part is zero)
  if (SPLIT == 1) {
#pragma unroll
    for (int c0 = 0; c0 < BN; c0 += 16) {
      if (!ok) break;
      uint32_t v[16];
      if (acc) tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + c0, v);
      if (row < ld) {
#pragma unroll
        for (int j = 0; j < 16; ++j)
          if (c0 + j < ncol) Y[(size_t)(col0 + c0 + j) * ld + row] = acc ? alpha * __uint_as_float(v[j]) : 0.0f;
      }
    }
  } else {
    // partial tile -> own shared memory (column-major, 128 rows per column; the ring is idle now)
    float* part = reinterpret_cast<float*>(smem);
#pragma unroll
    for (int c0 = 0; c0 < BN; c0 += 16) {
      uint32_t v[16];
      if (ok && acc) tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + c0, v);
#pragma unroll
      for (int j = 0; j < 16; ++j) part[(c0 + j) * BM + r_local] = ok && acc ? __uint_as_float(v[j]) : 0.0f;
    }
    cluster_sync();
    constexpr int CPR = BN / SPLIT;  // columns reduced by this CTA
    uint32_t peer[SPLIT];
    const uint32_t mine = smem_u32(part + split * CPR * BM + r_local);
#pragma unroll
    for (int p = 0; p < SPLIT; ++p) peer[p] = map_peer(mine, (uint32_t)p);
    // remote loads in groups of 32 issued back to back (they are independent), then each column is
    // summed over the partials in rank order
    constexpr int JG = 32 / SPLIT;  // columns per group
#pragma unroll
    for (int j0 = 0; j0 < CPR; j0 += JG) {
      float v[JG][SPLIT];
#pragma unroll
      for (int j = 0; j < JG; ++j)
#pragma unroll
        for (int p = 0; p < SPLIT; ++p) v[j][p] = ld_cluster(peer[p] + (uint32_t)((j0 + j) * BM * 4));
#pragma unroll
      for (int j = 0; j < JG; ++j) {
        const int c = split * CPR + j0 + j;
        float acc = 0.0f;
#pragma unroll
        for (int p = 0; p < SPLIT; ++p) acc += v[j][p];
        if (row < ld && c < ncol) Y[(size_t)(col0 + c) * ld + row] = alpha * acc;
      }
    }
    cluster_sync();  // no CTA leaves while a peer still reads its partial tile
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (threadIdx.x == 0 && !ok) {
    // a wait gave up: let the copies already issued land (bounded) before the CTA exits
    for (int kc = *s_consumed; kc < *s_issued; ++kc) mbar_wait(full0 + 8 * (kc % STAGES), (kc / STAGES) & 1, err);
  }
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    else
      (void)cudaGetLastError();
  });
  return fn;
}

CUtensorMap make_map(const float* base, int rank, const cuuint64_t* dims, const cuuint64_t* strides,
                     const cuuint32_t* box) {
  CUtensorMap m;
  auto fn = encode_fn();
  if (!fn) fail(DG_ERR_CUDA, "cuTensorMapEncodeTiled is unavailable");
  const cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, rank, (void*)base, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) fail(DG_ERR_CUDA, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
  return m;
}

}  // namespace

bool tc_gemm_available() { return encode_fn() != nullptr; }

std::vector<int> tc_gemm_splits(int ld) {
  std::vector<int> out;
  for (int split = 1; split <= 8; split *= 2)
    if (split == 1 || (ld / BK) / split >= 4) out.push_back(split);
  return out;
}

namespace {

template <int BN>
void set_smem_attributes() {
  // kernel attributes are per device
  static std::mutex mu;
  static std::set<int> done;
  int dev = 0;
  DG_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(mu);
  if (done.count(dev)) return;
  constexpr int S = TcShape<BN>::SMEM_BYTES;
  DG_CUDA(cudaFuncSetAttribute(tc_gemm_kernel<1, BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, S));
  DG_CUDA(cudaFuncSetAttribute(tc_gemm_kernel<2, BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, S));
  DG_CUDA(cudaFuncSetAttribute(tc_gemm_kernel<4, BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, S));
  DG_CUDA(cudaFuncSetAttribute(tc_gemm_kernel<8, BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, S));
  done.insert(dev);
}

template <int BN>
void launch_tc(const float* inv, int n_classes, const float* X, float* Y, int ld, int n_cols, const int4* d_tiles,
               int n_tiles, const int* d_kchunks, int* err, float alpha, cudaStream_t s, int split) {
  using SH = TcShape<BN>;
  const cuuint64_t dA[3] = {(cuuint64_t)ld, (cuuint64_t)ld, (cuuint64_t)n_classes};
  const cuuint64_t sAr[2] = {(cuuint64_t)ld * 4, (cuuint64_t)ld * ld * 4};
  const cuuint32_t bA[3] = {BK, BM, 1};
  const cuuint64_t dB[2] = {(cuuint64_t)ld, (cuuint64_t)n_cols};
  const cuuint64_t sBr[1] = {(cuuint64_t)ld * 4};
  const cuuint32_t bB[2] = {BK, BN};
  const CUtensorMap mA = make_map(inv, 3, dA, sAr, bA);
  const CUtensorMap mB = make_map(X, 2, dB, sBr, bB);
  set_smem_attributes<BN>();
  // Default: split K over a cluster of `split` CTAs so that the launch fills one wave of the
  // co-resident CTAs, keeping >= 4 K chunks each.
  const int nk = ld / BK;
  if (split == 0) {
    split = 1;
    while (split < 8 && n_tiles * split * 2 <= SH::SLOTS && nk / (split * 2) >= 4) split *= 2;
  }
  DG_REQUIRE(split == 1 || split == 2 || split == 4 || split == 8, "GEMM split must be 1, 2, 4 or 8");
  DG_REQUIRE(split == 1 || nk / split >= 1, "GEMM split larger than the K chunks");
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(n_tiles * split);
  cfg.blockDim = dim3(128);
  cfg.dynamicSmemBytes = SH::SMEM_BYTES;
  cfg.stream = s;
  cudaLaunchAttribute at[2];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  at[1].id = cudaLaunchAttributeClusterDimension;
  at[1].val.clusterDim.x = split;
  at[1].val.clusterDim.y = 1;
  at[1].val.clusterDim.z = 1;
  const bool pdl = pdl_enabled();
  cfg.attrs = pdl ? at : at + 1;
  cfg.numAttrs = (pdl ? 1 : 0) + (split == 1 ? 0 : 1);
  if (split == 1) DG_CUDA(cudaLaunchKernelEx(&cfg, tc_gemm_kernel<1, BN>, mA, mB, Y, ld, d_tiles, d_kchunks, err, alpha));
  else if (split == 2) DG_CUDA(cudaLaunchKernelEx(&cfg, tc_gemm_kernel<2, BN>, mA, mB, Y, ld, d_tiles, d_kchunks, err, alpha));
  else if (split == 4) DG_CUDA(cudaLaunchKernelEx(&cfg, tc_gemm_kernel<4, BN>, mA, mB, Y, ld, d_tiles, d_kchunks, err, alpha));
  else DG_CUDA(cudaLaunchKernelEx(&cfg, tc_gemm_kernel<8, BN>, mA, mB, Y, ld, d_tiles, d_kchunks, err, alpha));
  DG_LAUNCHED(1);
}

}  // namespace

void launch_class_gemm_tc(const float* inv, int n_classes, const float* X, float* Y, int ld, int n_cols,
                          const int4* d_tiles, int n_tiles, const int* d_kchunks, int* err, float alpha,
                          cudaStream_t s, int split, int bn) {
  if (n_tiles == 0) return;
  DG_REQUIRE(ld % BK == 0, "tensor-core GEMM needs a 32-aligned subdomain stride");
  DG_REQUIRE(bn == 64 || bn == 128 || bn == 256, "tensor-core GEMM tile width must be 64, 128 or 256");
  if (bn == 256) launch_tc<256>(inv, n_classes, X, Y, ld, n_cols, d_tiles, n_tiles, d_kchunks, err, alpha, s, split);
  else if (bn == 128)
    launch_tc<128>(inv, n_classes, X, Y, ld, n_cols, d_tiles, n_tiles, d_kchunks, err, alpha, s, split);
  else launch_tc<64>(inv, n_classes, X, Y, ld, n_cols, d_tiles, n_tiles, d_kchunks, err, alpha, s, split);
}

}  // namespace dg
