// pipe_probe.cu -- what one warp instruction of each class costs the SM's pipes.
//
// The evolve kernel's roofline counts issue slots; this probe checks that count
// against the hardware.  Each kernel below repeats one instruction class (eight
// independent chains per thread, so latency is hidden) and nothing else but the
// loop; under ncu the counters sm__inst_executed_pipe_<p> and
// sm__pipe_<p>_cycles_active give the pipe each class runs on and the cycles one
// warp instruction keeps it busy.  Build and profile (one GPU):
//
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 pipe_probe.cu -o pipe_probe
//   ncu --clock-control none --metrics <pipe counters> -k regex:probe --csv pipe_probe
//
// The probe prints only the order of its launches; every launch is in bounds by
// construction (one output word per thread, one cycle count per block).
#include <cstdio>
#include <cuda_runtime.h>
#include <stdint.h>

#define ITER 4096

template <int MODE>
__global__ void __launch_bounds__(256) probe(uint32_t *out, uint32_t seed)
{
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t u[8];
    float f[8];
    float2 p[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        u[i] = seed ^ (t * 2654435761u + i);
        f[i] = (float)(u[i] & 1023) * 1e-3f;
        p[i] = make_float2(f[i], f[i] + 1.0f);
    }
    const float a = 0.999f, b = 1e-4f;
#pragma unroll 1
    for (int it = 0; it < ITER; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            if (MODE == 0) asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(f[i]) : "f"(a), "f"(b));
            if (MODE == 1) p[i] = __ffma2_rn(p[i], make_float2(a, a), make_float2(b, b));
            if (MODE == 2) asm volatile("mul.lo.u32 %0, %0, %1;" : "+r"(u[i]) : "r"(0xD2511F53u));
            if (MODE == 3) {   // the 32x32 -> 64-bit product of a Philox round, both halves used
                const uint64_t w = (uint64_t)0xD2511F53u * u[i];
                u[i] = (uint32_t)(w >> 32) ^ (uint32_t)w;
            }
            if (MODE == 4) asm volatile("mul.hi.u32 %0, %0, %1;" : "+r"(u[i]) : "r"(0xD2511F53u));
            if (MODE == 5) asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(u[i]) : "r"(0x9E3779B9u), "r"(seed));
            if (MODE == 6) asm volatile("add.u32 %0, %0, %1;" : "+r"(u[i]) : "r"(0x9E3779B9u));
            if (MODE == 7) {
                float v;
                asm volatile("cvt.rn.f32.u32 %0, %1;" : "=f"(v) : "r"(u[i]));
                u[i] ^= __float_as_uint(v);
            }
            if (MODE == 8) asm volatile("ex2.approx.ftz.f32 %0, %0;" : "+f"(f[i]));
            if (MODE == 9) asm volatile("max.f32 %0, %0, %1;" : "+f"(f[i]) : "f"(a));
            if (MODE == 10) asm volatile("add.f32 %0, %0, %1;" : "+f"(f[i]) : "f"(b));
            if (MODE == 11) p[i] = __fadd2_rn(p[i], make_float2(b, b));
            if (MODE == 12) asm volatile("shr.u32 %0, %0, 1;" : "+r"(u[i]));
        }
    }
    uint32_t acc = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) acc ^= u[i] ^ __float_as_uint(f[i]) ^ __float_as_uint(p[i].x) ^ __float_as_uint(p[i].y);
    out[t] = acc;
}

static const char *names[] = {"FFMA",          "FFMA2 (packed pair)", "IMUL.LO", "IMAD.WIDE + xor",
                              "IMUL.HI",       "LOP3",                "IADD",    "I2F + xor",
                              "MUFU.EX2",      "FMNMX",               "FADD",    "FADD2 (packed pair)",
                              "SHF"};

template <int M> bool run(int blocks, uint32_t *out)
{
    probe<M><<<blocks, 256>>>(out, 12345u);
    const cudaError_t e = cudaDeviceSynchronize();
    printf("launch %2d: %s%s\n", M, names[M], e == cudaSuccess ? "" : " (failed)");
    return e == cudaSuccess;
}

int main()
{
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0) != cudaSuccess) return 1;
    const int blocks = sms * 4;   // 32 warps per SM
    uint32_t *out = nullptr;
    if (cudaMalloc(&out, (size_t)blocks * 256 * sizeof(uint32_t)) != cudaSuccess) return 1;
    const bool ok = run<0>(blocks, out) && run<1>(blocks, out) && run<2>(blocks, out) && run<3>(blocks, out) &&
                    run<4>(blocks, out) && run<5>(blocks, out) && run<6>(blocks, out) && run<7>(blocks, out) &&
                    run<8>(blocks, out) && run<9>(blocks, out) && run<10>(blocks, out) && run<11>(blocks, out) &&
                    run<12>(blocks, out);
    cudaFree(out);
    return ok ? 0 : 1;
}
