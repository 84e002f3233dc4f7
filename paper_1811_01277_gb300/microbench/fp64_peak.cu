// FP64 pipe throughput on the local GPU: DFMA (8 independent chains per
// thread), the f64 mma.sync shape m8n8k4, and kernels that issue both from
// the same warps (to see whether the FP64 tensor path and DFMA share one
// unit), and the bf16 / int8 mma.sync rates.  Each test runs for about target_s seconds so that clocks settle.
// Prints one line per test: name, TFLOP/s, seconds.
#include <cstdio>
#include <cstdlib>
#include <cuda_runtime.h>

__global__ void dfma8(double *out, long long iters, double x, double y)
{
    double a[8];
#pragma unroll
    for (int c = 0; c < 8; c++) a[c] = threadIdx.x * 1e-3 + c;
    for (long long i = 0; i < iters; i++) {
#pragma unroll
        for (int c = 0; c < 8; c++) a[c] = fma(a[c], x, y);
    }
    double s = 0;
#pragma unroll
    for (int c = 0; c < 8; c++) s += a[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void dmma_m8n8k4(double *out, long long iters)
{
    double a = 1.0 + threadIdx.x * 1e-6, b = 0.5, c[4][2];
#pragma unroll
    for (int k = 0; k < 4; k++) { c[k][0] = k; c[k][1] = k + 1; }
    for (long long i = 0; i < iters; i++) {
#pragma unroll
        for (int k = 0; k < 4; k++)
            asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
                         : "+d"(c[k][0]), "+d"(c[k][1]) : "d"(a), "d"(b));
    }
    double s = 0;
#pragma unroll
    for (int k = 0; k < 4; k++) s += c[k][0] + c[k][1];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Per iteration every thread issues 8 DFMA (16 flops; 512 per warp) and the
// warp issues NM m8n8k4 f64 MMAs (512 flops each).  If the tensor path had
// its own FP64 units the sum would exceed the DFMA-only rate.
template <int NM>
__global__ void dfma_dmma_mix(double *out, long long iters, double x, double y)
{
    double a[8], ma = 1.0 + threadIdx.x * 1e-6, mb = 0.5, c[NM][2];
#pragma unroll
    for (int k = 0; k < 8; k++) a[k] = threadIdx.x * 1e-3 + k;
#pragma unroll
    for (int k = 0; k < NM; k++) { c[k][0] = k; c[k][1] = k + 1; }
    for (long long i = 0; i < iters; i++) {
#pragma unroll
        for (int k = 0; k < 8; k++) a[k] = fma(a[k], x, y);
#pragma unroll
        for (int k = 0; k < NM; k++)
            asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
                         : "+d"(c[k][0]), "+d"(c[k][1]) : "d"(ma), "d"(mb));
    }
    double s = 0;
#pragma unroll
    for (int k = 0; k < 8; k++) s += a[k];
#pragma unroll
    for (int k = 0; k < NM; k++) s += c[k][0] + c[k][1];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Half the warps of a block run DFMA chains, the other half m8n8k4 MMAs.
__global__ void dfma_dmma_split(double *out, long long iters_f, long long iters_m, double x, double y)
{
    double s = 0;
    if ((threadIdx.x >> 5) & 1) {
        double ma = 1.0 + threadIdx.x * 1e-6, mb = 0.5, c[4][2];
#pragma unroll
        for (int k = 0; k < 4; k++) { c[k][0] = k; c[k][1] = k + 1; }
        for (long long i = 0; i < iters_m; i++) {
#pragma unroll
            for (int k = 0; k < 4; k++)
                asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
                             : "+d"(c[k][0]), "+d"(c[k][1]) : "d"(ma), "d"(mb));
        }
#pragma unroll
        for (int k = 0; k < 4; k++) s += c[k][0] + c[k][1];
    } else {
        double a[8];
#pragma unroll
        for (int k = 0; k < 8; k++) a[k] = threadIdx.x * 1e-3 + k;
        for (long long i = 0; i < iters_f; i++) {
#pragma unroll
            for (int k = 0; k < 8; k++) a[k] = fma(a[k], x, y);
        }
#pragma unroll
        for (int k = 0; k < 8; k++) s += a[k];
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}


// Legacy warp-level tensor path (mma.sync), for the FP64-emulation design:
// 8 independent accumulator chains per warp.
__global__ void hmma_bf16(float *out, long long iters)
{
    unsigned a[4], b[2];
#pragma unroll
    for (int i = 0; i < 4; i++) a[i] = 0x3f803f80u ^ (threadIdx.x << 3);
    b[0] = 0x3f003f00u;
    b[1] = 0x3e803e80u;
    float c[8][4];
#pragma unroll
    for (int k = 0; k < 8; k++)
#pragma unroll
        for (int i = 0; i < 4; i++) c[k][i] = 0.f;
    for (long long it = 0; it < iters; it++) {
#pragma unroll
        for (int k = 0; k < 8; k++)
            asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
                         : "+f"(c[k][0]), "+f"(c[k][1]), "+f"(c[k][2]), "+f"(c[k][3])
                         : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 8; k++) s += c[k][0] + c[k][1] + c[k][2] + c[k][3];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void imma_s8(int *out, long long iters)
{
    unsigned a[4], b[2];
#pragma unroll
    for (int i = 0; i < 4; i++) a[i] = 0x01020304u ^ threadIdx.x;
    b[0] = 0x05060708u;
    b[1] = 0x0102fefdu;
    int c[8][4];
#pragma unroll
    for (int k = 0; k < 8; k++)
#pragma unroll
        for (int i = 0; i < 4; i++) c[k][i] = 0;
    for (long long it = 0; it < iters; it++) {
#pragma unroll
        for (int k = 0; k < 8; k++)
            asm volatile("mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
                         : "+r"(c[k][0]), "+r"(c[k][1]), "+r"(c[k][2]), "+r"(c[k][3])
                         : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
    }
    int s = 0;
#pragma unroll
    for (int k = 0; k < 8; k++) s += c[k][0] + c[k][1] + c[k][2] + c[k][3];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

static cudaEvent_t e0, e1;

template <class F>
static float timed(F launch)
{
    float ms = 0;
    cudaEventRecord(e0);
    launch();
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    return ms;
}

// Calibrates the iteration count on a short run, then times about target_s.
template <class F>
static void run(const char *name, double target_s, double flops_per_iter, F launch_with_iters)
{
    long long it = 100;
    launch_with_iters(it);
    float ms = timed([&] { launch_with_iters(it); });
    it = (long long)(it * target_s * 1000.0 / (ms > 0.01f ? ms : 0.01f));
    if (it < 1) it = 1;
    ms = timed([&] { launch_with_iters(it); });
    printf("%s %.4f %.3f\n", name, flops_per_iter * it / (ms * 1e-3) / 1e12, ms * 1e-3);
}

int main(int argc, char **argv)
{
    double target_s = argc > 1 ? atof(argv[1]) : 1.0;
    cudaDeviceProp p;
    if (cudaGetDeviceProperties(&p, 0) != cudaSuccess) { printf("no device\n"); return 1; }
    const int grid = p.multiProcessorCount * 8;
    double *out;
    if (cudaMalloc(&out, sizeof(double) * grid * 256) != cudaSuccess) return 1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const double X = 1.0000001, Y = 1e-9;

    run("dfma", target_s, 16.0 * grid * 256,
        [&](long long it) { dfma8<<<grid, 256>>>(out, it, X, Y); });
    run("dmma_m8n8k4", target_s, 512.0 * 4 * grid * 4,
        [&](long long it) { dmma_m8n8k4<<<grid, 128>>>(out, it); });
    // 8 warps per block: 8 x 512 DFMA flops + NM x 8 x 512 MMA flops per iteration
    run("mix_dfma_dmma1", target_s, (512.0 + 512.0 * 1) * 8 * grid,
        [&](long long it) { dfma_dmma_mix<1><<<grid, 256>>>(out, it, X, Y); });
    run("mix_dfma_dmma2", target_s, (512.0 + 512.0 * 2) * 8 * grid,
        [&](long long it) { dfma_dmma_mix<2><<<grid, 256>>>(out, it, X, Y); });
    // split warps: DFMA warps run 4x the iterations of MMA warps so both take
    // about the same time alone (8 chains x 512 flops vs 4 MMAs x 512 flops)
    run("split_dfma_dmma", target_s, (4.0 * 512.0 + 4.0 * 512.0) * 4 * grid,
        [&](long long it) { dfma_dmma_split<<<grid, 256>>>(out, 4 * it, it, X, Y); });
    // 8 warps per block, 8 MMAs per warp and iteration
    run("hmma_bf16_m16n8k16", target_s, 4096.0 * 8 * 8 * grid,
        [&](long long it) { hmma_bf16<<<grid, 256>>>((float *)out, it); });
    run("imma_s8_m16n8k32", target_s, 8192.0 * 8 * 8 * grid,
        [&](long long it) { imma_s8<<<grid, 256>>>((int *)out, it); });
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) { printf("cuda error %s\n", cudaGetErrorString(e)); return 1; }
    return 0;
}
