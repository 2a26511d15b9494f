// Tensor-core issue-rate probe (test infrastructure, not part of the library): one CTA per SM
// issues back-to-back tcgen05.mma (kind::f16, K = 16, BF16, float32 accumulator) on fixed
// 128-byte-swizzled K-major operand tiles in shared memory, without TMA traffic, and times them
// with clock64.  It first checks that an A operand copied into TMEM with tcgen05.cp gives the
// same product as A read from shared memory, then reports cycles per MMA for: 128x128 from
// shared memory; A from TMEM; 128x256; 128x128 into two and four accumulators in turn; 128x64;
// and 128x128 issued from two warps (on the same tiles, and each on its own) and from two lanes
// of one warp.  Every wait is bounded; a timeout is reported, not hung on.
// Output: one line per form, "<form> grid <g>: <c> cycles per MMA (nominal <n>), ...".
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>
#include <cmath>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

__device__ __forceinline__ uint32_t su32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4);
  d |= static_cast<uint64_t>(1u) << 16;
  d |= static_cast<uint64_t>(1024u >> 4) << 32;
  d |= static_cast<uint64_t>(1u) << 46;
  d |= static_cast<uint64_t>(2u) << 61;
  return d;
}
__host__ __device__ constexpr uint32_t idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<uint32_t>(N >> 3) << 17) |
         (static_cast<uint32_t>(M >> 4) << 24);
}
__device__ __forceinline__ void mma_ss(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
               "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
               "l"(a), "l"(b), "r"(id), "r"(acc));
}
__device__ __forceinline__ void mma_ts(uint32_t d, uint32_t a, uint64_t b, uint32_t id, uint32_t acc) {
  asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
               "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d),
               "r"(a), "l"(b), "r"(id), "r"(acc));
}
__device__ __forceinline__ void cp_128x256b(uint32_t taddr, uint64_t s) {
  asm volatile("tcgen05.cp.cta_group::1.128x256b [%0], %1;" ::"r"(taddr), "l"(s));
}
__device__ __forceinline__ void commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar)) : "memory");
}
__device__ __forceinline__ bool wait(uint64_t *bar, uint32_t ph) {
  const long long t0 = clock64();
  while (true) {
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok) : "r"(su32(bar)), "r"(ph) : "memory");
    if (ok) return true;
    if (clock64() - t0 > 2000000000LL) return false;
  }
}

__global__ void __launch_bounds__(128, 1) probe(int mode, int iters, const __nv_bfloat16 *gA,
                                                const __nv_bfloat16 *gB, float *out,
                                                long long *cyc, int *err) {
  extern __shared__ uint8_t raw[];
  uint8_t *sm = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(raw) + 1023) & ~uintptr_t(1023));
  uint8_t *sA = sm;                 // 128 rows x 128 B
  uint8_t *sB = sm + 16384;         // 256 rows x 128 B
  uint8_t *sA2 = sm + 16384 + 32768;  // a copy of A at its own address (mode 9)
  uint64_t *bar = reinterpret_cast<uint64_t *>(sm + 16384 + 32768 + 16384);
  uint32_t *slot = reinterpret_cast<uint32_t *>(bar + 2);
  const int t = threadIdx.x;
  // swizzled K-major fill: element (r, k), k < 64: byte r*128 + (((2k)/16) ^ (r%8))*16 + (2k)%16
  for (int idx = t; idx < 128 * 64; idx += 128) {
    const int r = idx / 64, k = idx % 64;
    const int off = r * 128 + ((((2 * k) / 16) ^ (r % 8)) * 16) + (2 * k) % 16;
    *reinterpret_cast<__nv_bfloat16 *>(sA + off) = gA[idx];
    *reinterpret_cast<__nv_bfloat16 *>(sA2 + off) = gA[idx];
  }
  for (int idx = t; idx < 256 * 64; idx += 128) {
    const int r = idx / 64, k = idx % 64;
    const int off = r * 128 + ((((2 * k) / 16) ^ (r % 8)) * 16) + (2 * k) % 16;
    *reinterpret_cast<__nv_bfloat16 *>(sB + off) = gB[idx];
  }
  if (t == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(bar)) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(bar + 1)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (t < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(su32(slot)) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t base = *slot;
  const uint64_t dA = sdesc(su32(sA)), dB = sdesc(su32(sB));
  // modes: 0 N=128, 1 N=128 A in TMEM, 2 N=256, 3 N=128 two accumulators, 4 N=128 four
  // accumulators, 5 N=256 two accumulators, 6 N=64
  const int N = (mode == 2 || mode == 5) ? 256 : (mode == 6 ? 64 : 128);
  const int nacc = mode == 3 ? 2 : (mode == 4 ? 4 : (mode == 5 ? 2 : 1));
  const uint32_t id = idesc(128, N);
  const uint32_t tA = base + 256;   // columns [256, 288): A's 4 K-steps x 8 columns
  bool ok = true;
  if (((mode == 7 || mode == 9) && (t == 0 || t == 32)) || (mode == 8 && (t == 0 || t == 1))) {
    // two issuing threads, each its own N = 128 accumulator: lane 0 of warps 0 and 1 (mode 7,
    // both on the same operand tiles; mode 9, each on its own two tiles) or lanes 0 and 1 of
    // warp 0 (mode 8)
    const bool second = mode == 8 ? t == 1 : t == 32;
    const uint32_t d = base + (second ? 128u : 0u);
    const uint64_t a = (mode == 9 && second) ? sdesc(su32(sA2)) : dA;
    const uint64_t b = (mode == 9 && second) ? sdesc(su32(sB + 16384)) : dB;
    const long long c0 = clock64();
    for (int it = 0; it < iters; ++it)
      for (int kk = 0; kk < 4; ++kk)
        mma_ss(d, a + 2u * kk, b + 2u * kk, idesc(128, 128), (it > 0 || kk > 0) ? 1u : 0u);
    commit(bar + (second ? 1 : 0));
    ok = wait(bar + (second ? 1 : 0), 0);
    if (t == 0) cyc[blockIdx.x] = clock64() - c0;
    if (!ok) atomicExch(err, 1);
  } else if (mode < 7 && t == 0) {
    if (mode == 1) {
      for (int kk = 0; kk < 4; ++kk) cp_128x256b(tA + 8 * kk, dA + 2u * kk);
      commit(bar + 1);
      ok = wait(bar + 1, 0);
    }
    const long long c0 = clock64();
    for (int it = 0; ok && it < iters; ++it) {
      for (int kk = 0; kk < 4; ++kk) {
        const int a = (it * 4 + kk) % nacc;
        const uint32_t acc = (it * 4 + kk >= nacc) ? 1u : 0u;
        const uint32_t d = base + static_cast<uint32_t>(a * (nacc == 2 && N == 256 ? 256 : 128));
        if (mode == 1) mma_ts(base, tA + 8 * kk, dB + 2u * kk, id, acc);
        else mma_ss(d, dA + 2u * kk, dB + 2u * kk, id, acc);
      }
    }
    if (ok) {
      commit(bar);
      ok = wait(bar, 0);
    }
    cyc[blockIdx.x] = clock64() - c0;
    if (!ok) atomicExch(err, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (blockIdx.x == 0 && *err == 0) {
    const int w = t / 32, l = t % 32;
    for (int c = 0; c < 128; c += 32) {
      uint32_t r[32];
      const uint32_t ta = base + (static_cast<uint32_t>(w * 32) << 16) + c;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
          "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
          "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
            "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
            "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
            "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
            "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
            "=r"(r[31])
          : "r"(ta));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      for (int j = 0; j < 32; ++j) out[(w * 32 + l) * 128 + c + j] = __uint_as_float(r[j]);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (t < 32) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(base) : "memory");
}

int main(int argc, char **argv) {
  const int grid = argc > 1 ? atoi(argv[1]) : 152;
  std::vector<__nv_bfloat16> hA(128 * 64), hB(256 * 64);
  std::vector<float> fA(128 * 64), fB(256 * 64);
  uint32_t s = 12345;
  auto rnd = [&]() { s = s * 1664525u + 1013904223u; return ((s >> 8) & 0xFFFF) / 32768.0f - 1.0f; };
  for (int i = 0; i < 128 * 64; ++i) { hA[i] = __float2bfloat16(rnd()); fA[i] = __bfloat162float(hA[i]); }
  for (int i = 0; i < 256 * 64; ++i) { hB[i] = __float2bfloat16(rnd()); fB[i] = __bfloat162float(hB[i]); }
  __nv_bfloat16 *dA, *dB; float *dOut; long long *dCyc; int *dErr;
  cudaMalloc(&dA, hA.size() * 2); cudaMalloc(&dB, hB.size() * 2);
  cudaMalloc(&dOut, 128 * 128 * 4); cudaMalloc(&dCyc, 1024 * 8); cudaMalloc(&dErr, 4);
  cudaMemcpy(dA, hA.data(), hA.size() * 2, cudaMemcpyHostToDevice);
  cudaMemcpy(dB, hB.data(), hB.size() * 2, cudaMemcpyHostToDevice);
  const size_t smem = 200 * 1024;   // one CTA per SM (the whole TMEM each)
  cudaFuncSetAttribute(probe, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  std::vector<float> ref(128 * 128);
  for (int r = 0; r < 128; ++r)
    for (int c = 0; c < 128; ++c) {
      double a = 0; for (int k = 0; k < 64; ++k) a += (double)fA[r * 64 + k] * fB[c * 64 + k];
      ref[r * 128 + c] = (float)a;
    }
  std::vector<float> res[2];
  for (int mode = 0; mode < 2; ++mode) {
    cudaMemset(dErr, 0, 4);
    probe<<<1, 128, smem>>>(mode, 1, dA, dB, dOut, dCyc, dErr);
    cudaError_t e = cudaDeviceSynchronize();
    int herr = 0; cudaMemcpy(&herr, dErr, 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess || herr) { printf("mode %d check: error %s / timeout %d\n", mode, cudaGetErrorString(e), herr); return 1; }
    res[mode].resize(128 * 128);
    cudaMemcpy(res[mode].data(), dOut, 128 * 128 * 4, cudaMemcpyDeviceToHost);
    double md = 0; for (int i = 0; i < 128 * 128; ++i) md = fmax(md, fabs(res[mode][i] - ref[i]));
    printf("mode %d (1 x K=64): max |D - ref| = %.3e\n", mode, md);
  }
  int same = 0; for (int i = 0; i < 128 * 128; ++i) same += (res[0][i] == res[1][i]);
  printf("TMEM-A vs smem-A: %d of %d elements bitwise equal\n", same, 128 * 128);
  const char *names[10] = {"A,B smem N=128", "A tmem, B smem N=128", "A,B smem N=256",
                           "N=128, 2 accumulators", "N=128, 4 accumulators", "N=256, 2 accumulators",
                           "N=64", "N=128, 2 issuing warps", "N=128, 2 lanes of a warp",
                           "N=128, 2 warps, own tiles"};
  for (int mode = 0; mode < 10; ++mode) {
    const int iters = 2000;
    cudaMemset(dErr, 0, 4);
    probe<<<grid, 128, smem>>>(mode, iters, dA, dB, dOut, dCyc, dErr);
    cudaError_t e = cudaDeviceSynchronize();
    int herr = 0; cudaMemcpy(&herr, dErr, 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess || herr) { printf("mode %d timing: error %s / timeout %d\n", mode, cudaGetErrorString(e), herr); return 1; }
    std::vector<long long> cyc(grid);
    cudaMemcpy(cyc.data(), dCyc, grid * 8, cudaMemcpyDeviceToHost);
    double avg = 0; for (auto c : cyc) avg += c; avg /= grid;
    const int N = (mode == 2 || mode == 5) ? 256 : (mode == 6 ? 64 : 128);
    const double per = avg / (iters * 4.0 * (mode >= 7 ? 2 : 1));
    printf("%-22s grid %d: %.1f cycles per MMA (nominal %d), %.0f flop/cycle/SM\n", names[mode], grid,
           per, N / 2, 2.0 * 128 * N * 16 / per);
  }
  return 0;
}
