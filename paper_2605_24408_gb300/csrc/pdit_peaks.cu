// On-chip peaks that bound the sweep kernels, measured on the device the
// library runs on: shared-memory load bandwidth (the binding roofline of the
// kernels that keep their working set in shared memory), the issue rates of
// 32-bit integer multiply-add and of the 8-bit dot product dp4a (the
// arithmetic of the influence sums and of the deferred table updates), and
// the rates of the warp-level tensor instructions for f16 and s8 operands.
//
// Each probe runs one CTA of 1024 threads per SM and measures both wall time
// (CUDA events) and SM cycles (clock64 around the timed loop, per CTA), so
// the figures come out per second and per clock per SM. The loads and the
// arithmetic are inline PTX marked volatile so that none of them is folded
// or hoisted out of the loop.
#include <cuda_runtime.h>

#include <algorithm>

#include "../../include/pdit.h"

namespace {

constexpr int kThreads = 1024;
constexpr int kSmemVecs = 8192;  // 128 KB of 16-byte vectors: one CTA per SM

// Every thread reads 16-byte vectors; the 32 lanes of a warp read 512
// contiguous bytes (four full wavefronts, no bank conflict); one pass of
// the CTA reads the whole 128 KB buffer. The addresses move by one warp's
// span every trip, so no load is invariant across the loop (a load with a
// fixed address could be hoisted out of it by the assembler).
__global__ void __launch_bounds__(kThreads) smem_probe_kernel(int iters, unsigned *sink,
                                                              unsigned long long *cycles) {
    extern __shared__ __align__(16) uint4 buf[];
    for (int k = threadIdx.x; k < kSmemVecs; k += blockDim.x)
        buf[k] = make_uint4(k, 3u * k + 1u, 5u * k + 2u, 7u * k + 3u);
    __syncthreads();
    const unsigned base = (unsigned)__cvta_generic_to_shared(buf);
    unsigned a0 = 0, a1 = 0, a2 = 0, a3 = 0;
    const unsigned long long t0 = clock64();
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kSmemVecs / kThreads; ++u) {
            const unsigned addr = base + 16u * ((unsigned)(threadIdx.x + kThreads * u + 32 * it) & (kSmemVecs - 1));
            unsigned x, y, z, w;
            asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                         : "=r"(x), "=r"(y), "=r"(z), "=r"(w)
                         : "r"(addr));
            a0 ^= x;
            a1 ^= y;
            a2 ^= z;
            a3 ^= w;
        }
    }
    __syncthreads();
    const unsigned long long t1 = clock64();
    if ((a0 ^ a1 ^ a2 ^ a3) == 0x9E3779B9u) sink[0] = 1u;  // keeps the loads live
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

// Eight independent dependency chains per thread of `dp4a.s32.s32` (OP 0) or
// `mad.lo.s32` (OP 1).
template <int OP>
__global__ void __launch_bounds__(kThreads) alu_probe_kernel(int iters, int *sink, unsigned long long *cycles) {
    int acc[8], a[8];
    const int b = (int)(threadIdx.x * 0x01010101u) | 0x01;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        acc[k] = k;
        a[k] = (int)(threadIdx.x + 0x01020304u * (unsigned)k);
    }
    __syncthreads();
    const unsigned long long t0 = clock64();
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                if constexpr (OP == 0)
                    asm volatile("dp4a.s32.s32 %0, %1, %2, %0;" : "+r"(acc[k]) : "r"(a[k]), "r"(b));
                else
                    asm volatile("mad.lo.s32 %0, %1, %2, %0;" : "+r"(acc[k]) : "r"(a[k]), "r"(b));
            }
        }
    }
    __syncthreads();
    const unsigned long long t1 = clock64();
    int s = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s ^= acc[k];
    if (s == 0x7F4A7C15) sink[0] = s;
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

// Four independent accumulator chains per warp of the legacy warp-level
// tensor instruction: OP 0 mma.sync m16n8k16 f16 x f16 -> f32 (2048 MACs),
// OP 1 mma.sync m16n8k32 s8 x s8 -> s32 (4096 MACs).
template <int OP>
__global__ void __launch_bounds__(kThreads) mma_probe_kernel(int iters, int *sink, unsigned long long *cycles) {
    const uint32_t a0 = 0x3C003C00u ^ threadIdx.x, a1 = a0 + 1, a2 = a0 + 2, a3 = a0 + 3;
    const uint32_t b0 = 0x3C003C00u ^ (threadIdx.x * 7u), b1 = b0 + 5;
    float f[4][4];
    int c[4][4];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            f[q][e] = 0.0f;
            c[q][e] = 0;
        }
    __syncthreads();
    const unsigned long long t0 = clock64();
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 2; ++u) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if constexpr (OP == 0)
                    asm volatile(
                        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, "
                        "{%8, %9}, {%0, %1, %2, %3};"
                        : "+f"(f[q][0]), "+f"(f[q][1]), "+f"(f[q][2]), "+f"(f[q][3])
                        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
                else
                    asm volatile(
                        "mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, "
                        "{%8, %9}, {%0, %1, %2, %3};"
                        : "+r"(c[q][0]), "+r"(c[q][1]), "+r"(c[q][2]), "+r"(c[q][3])
                        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
            }
        }
    }
    __syncthreads();
    const unsigned long long t1 = clock64();
    int sacc = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int e = 0; e < 4; ++e) sacc ^= c[q][e] ^ __float_as_int(f[q][e]);
    if (sacc == 0x2545F491) sink[0] = sacc;
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

struct Timing {
    double seconds;
    double cycles;  // mean over CTAs
};

template <typename Launch>
int time_probe(Launch launch, int sms, unsigned long long *dcyc, cudaStream_t st, Timing *out) {
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return PDIT_ECUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return PDIT_ECUDA;
    }
    int rc = PDIT_OK;
    float ms = 0.0f;
    launch(1);  // warm-up: module load, clocks up
    if (cudaEventRecord(e0, st) != cudaSuccess) rc = PDIT_ECUDA;
    if (!rc) launch(0);
    if (!rc && cudaEventRecord(e1, st) != cudaSuccess) rc = PDIT_ECUDA;
    if (!rc && cudaGetLastError() != cudaSuccess) rc = PDIT_ECUDA;
    if (!rc && cudaEventSynchronize(e1) != cudaSuccess) rc = PDIT_ECUDA;
    if (!rc && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) rc = PDIT_ECUDA;
    if (!rc) {
        unsigned long long *h = new unsigned long long[sms];
        if (cudaMemcpy(h, dcyc, sizeof(unsigned long long) * sms, cudaMemcpyDeviceToHost) != cudaSuccess) {
            rc = PDIT_ECUDA;
        } else {
            double c = 0.0;
            for (int k = 0; k < sms; ++k) c += (double)h[k];
            out->cycles = c / sms;
            out->seconds = ms / 1000.0;
        }
        delete[] h;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

}  // namespace

extern "C" int pdit_probe_peaks(int iters, double *out) {
    if (iters < 1 || !out) return PDIT_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PDIT_ECUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return PDIT_ECUDA;
    const size_t smem = sizeof(uint4) * kSmemVecs;
    if (cudaFuncSetAttribute(smem_probe_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return PDIT_ECUDA;
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return PDIT_ECUDA;
    void *dsink = nullptr;
    unsigned long long *dcyc = nullptr;
    int rc = PDIT_OK;
    if (cudaMalloc(&dsink, 16) != cudaSuccess || cudaMalloc(&dcyc, sizeof(unsigned long long) * sms) != cudaSuccess)
        rc = PDIT_ENOMEM;
    Timing t{};
    if (!rc) {
        rc = time_probe([&](int warm) {
            smem_probe_kernel<<<sms, kThreads, smem, st>>>(warm ? 4 : iters, (unsigned *)dsink, dcyc);
        }, sms, dcyc, st, &t);
        if (!rc) {
            const double bytes = (double)iters * kSmemVecs * sizeof(uint4);  // per CTA = per SM
            out[0] = bytes * sms / t.seconds;
            out[1] = bytes / t.cycles;
        }
    }
    if (!rc) {
        rc = time_probe([&](int warm) {
            alu_probe_kernel<0><<<sms, kThreads, 0, st>>>(warm ? 4 : iters, (int *)dsink, dcyc);
        }, sms, dcyc, st, &t);
        if (!rc) {
            const double ops = (double)iters * 32.0 * kThreads;  // per SM
            out[2] = ops * sms / t.seconds;
            out[3] = ops / t.cycles;
        }
    }
    if (!rc) {
        rc = time_probe([&](int warm) {
            alu_probe_kernel<1><<<sms, kThreads, 0, st>>>(warm ? 4 : iters, (int *)dsink, dcyc);
        }, sms, dcyc, st, &t);
        if (!rc) {
            const double ops = (double)iters * 32.0 * kThreads;
            out[4] = ops * sms / t.seconds;
            out[5] = ops / t.cycles;
        }
    }
    for (int op = 0; op < 2 && !rc; ++op) {
        rc = time_probe([&](int warm) {
            if (op == 0)
                mma_probe_kernel<0><<<sms, kThreads, 0, st>>>(warm ? 4 : iters, (int *)dsink, dcyc);
            else
                mma_probe_kernel<1><<<sms, kThreads, 0, st>>>(warm ? 4 : iters, (int *)dsink, dcyc);
        }, sms, dcyc, st, &t);
        if (!rc) {
            // warps per SM x instructions per warp x MACs per instruction
            const double macs = (double)iters * 8.0 * (kThreads / 32) * (op == 0 ? 2048.0 : 4096.0);
            out[6 + 2 * op] = macs * sms / t.seconds;
            out[7 + 2 * op] = macs / t.cycles;
        }
    }
    if (dsink) cudaFree(dsink);
    if (dcyc) cudaFree(dcyc);
    cudaStreamDestroy(st);
    return rc;
}
