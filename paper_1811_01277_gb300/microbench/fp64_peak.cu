// FP64 pipe throughput on the local GPU: DFMA (8 independent chains per
// thread) and the f64 mma.sync shapes, each run for about a second so that
// clocks settle.  Prints one line per test: name, TFLOP/s, seconds.
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

int main(int argc, char **argv)
{
    double target_s = argc > 1 ? atof(argv[1]) : 1.0;
    cudaDeviceProp p;
    if (cudaGetDeviceProperties(&p, 0) != cudaSuccess) { printf("no device\n"); return 1; }
    const int sms = p.multiProcessorCount, block = 256, grid = sms * 8;
    double *out;
    if (cudaMalloc(&out, sizeof(double) * grid * block) != cudaSuccess) return 1;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float ms;
    // calibrate then run for ~target_s
    long long it = 1000;
    dfma8<<<grid, block>>>(out, it, 1.0000001, 1e-9);
    cudaEventRecord(e0);
    dfma8<<<grid, block>>>(out, it, 1.0000001, 1e-9);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    it = (long long)(it * target_s * 1000.0 / ms);
    cudaEventRecord(e0);
    dfma8<<<grid, block>>>(out, it, 1.0000001, 1e-9);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    printf("dfma %.4f %.3f sms=%d\n", 2.0 * 8 * it * (double)grid * block / (ms * 1e-3) / 1e12, ms * 1e-3, sms);
    long long jt = 200;
    dmma_m8n8k4<<<grid, 128>>>(out, jt);
    cudaEventRecord(e0);
    dmma_m8n8k4<<<grid, 128>>>(out, jt);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    jt = (long long)(jt * target_s * 1000.0 / ms);
    cudaEventRecord(e0);
    dmma_m8n8k4<<<grid, 128>>>(out, jt);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    printf("dmma_m8n8k4 %.4f %.3f\n", 512.0 * 4 * jt * grid * 4.0 / (ms * 1e-3) / 1e12, ms * 1e-3);
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) { printf("cuda error %s\n", cudaGetErrorString(e)); return 1; }
    return 0;
}
