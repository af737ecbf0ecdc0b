// Stand-alone micro-benchmark of the fused step's memory access pattern (not
// part of the library): every thread reads the Q populations of f and of g of
// its node and writes them back, for a 256 x 256 x 1024 D3Q19 grid, in two
// orders (grid-stride, and 32 x 8 tiles marching along z as the fused step
// does) and two layouts (population-major planes, 32-node blocks), at float32
// and float16.  Prints ms per pass and GB/s of the algorithmic bytes.
#include <cstdio>
#include <cstdint>
#include <cuda_runtime.h>
#include <cuda_fp16.h>
constexpr int Q = 19;
template <class T, bool BLK>
__device__ __forceinline__ int64_t idx(int a, int64_t node, int64_t N) {
    return BLK ? ((node >> 5) * Q + a) * 32 + (node & 31) : a * N + node;
}
// plain: grid-stride over nodes in order
template <class T, bool BLK>
__global__ void __launch_bounds__(256) k_plain(const T* __restrict__ f, const T* __restrict__ g, T* __restrict__ fo, T* __restrict__ go, int64_t N) {
    for (int64_t node = blockIdx.x * 256ll + threadIdx.x; node < N; node += int64_t(gridDim.x) * 256) {
        T vf[Q], vg[Q];
#pragma unroll
        for (int a = 0; a < Q; ++a) { vf[a] = f[idx<T,BLK>(a, node, N)]; vg[a] = g[idx<T,BLK>(a, node, N)]; }
#pragma unroll
        for (int a = 0; a < Q; ++a) { fo[idx<T,BLK>(a, node, N)] = vf[a]; go[idx<T,BLK>(a, node, N)] = vg[a]; }
    }
}
// march: persistent blocks own 32x8 tiles and march along z (like the fused step)
template <class T, bool BLK>
__global__ void __launch_bounds__(256, 3) k_march(const T* __restrict__ f, const T* __restrict__ g, T* __restrict__ fo, T* __restrict__ go,
                                               int nx, int ny, int nz, int seglen) {
    const int tiles_x = nx / 32, tiles_y = ny / 8, ntiles = tiles_x * tiles_y, nseg = nz / seglen;
    const int64_t N = int64_t(nx) * ny * nz;
    for (int item = blockIdx.x; item < ntiles * nseg; item += gridDim.x) {
        const int tile = item % ntiles, seg = item / ntiles;
        const int x = (tile % tiles_x) * 32 + threadIdx.x, y = (tile / tiles_x) * 8 + threadIdx.y;
        for (int z = seg * seglen; z < (seg + 1) * seglen; ++z) {
            const int64_t node = (int64_t(z) * ny + y) * nx + x;
            T vf[Q], vg[Q];
#pragma unroll
            for (int a = 0; a < Q; ++a) { vf[a] = f[idx<T,BLK>(a, node, N)]; vg[a] = g[idx<T,BLK>(a, node, N)]; }
#pragma unroll
            for (int a = 0; a < Q; ++a) { fo[idx<T,BLK>(a, node, N)] = vf[a]; go[idx<T,BLK>(a, node, N)] = vg[a]; }
        }
    }
}
template <class T, bool BLK, bool MARCH>
float run(void* f, void* g, void* fo, void* go, int nx, int ny, int nz, int sms) {
    cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
    const int64_t N = int64_t(nx) * ny * nz;
    auto launch = [&]() {
        if (MARCH) k_march<T,BLK><<<sms * 3, dim3(32, 8)>>>((T*)f, (T*)g, (T*)fo, (T*)go, nx, ny, nz, 64);
        else k_plain<T,BLK><<<sms * 4, 256>>>((T*)f, (T*)g, (T*)fo, (T*)go, N);
    };
    for (int i = 0; i < 3; ++i) launch();
    cudaEventRecord(e0);
    const int K = 20;
    for (int i = 0; i < K; ++i) launch();
    cudaEventRecord(e1); cudaEventSynchronize(e1);
    float ms; cudaEventElapsedTime(&ms, e0, e1);
    const double bytes = 4.0 * Q * sizeof(T) * N;
    printf("%s %s %s: %.3f ms  %.0f GB/s\n", sizeof(T) == 4 ? "f32" : "f16", BLK ? "blocked" : "planar ", MARCH ? "march" : "plain",
           ms / K, bytes / (ms / K * 1e-3) / 1e9);
    return ms;
}
int main() {
    const int nx = 256, ny = 256, nz = 1024;
    const int64_t N = int64_t(nx) * ny * nz;
    int sms; cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
    void *f, *g, *fo, *go;
    const size_t bytes = size_t(N) * Q * 4;
    if (cudaMalloc(&f, bytes) || cudaMalloc(&g, bytes) || cudaMalloc(&fo, bytes) || cudaMalloc(&go, bytes)) { printf("alloc failed\n"); return 1; }
    cudaMemset(f, 0, bytes); cudaMemset(g, 0, bytes);
    run<float, false, false>(f, g, fo, go, nx, ny, nz, sms);
    run<float, true, false>(f, g, fo, go, nx, ny, nz, sms);
    run<float, false, true>(f, g, fo, go, nx, ny, nz, sms);
    run<float, true, true>(f, g, fo, go, nx, ny, nz, sms);
    run<__half, false, false>(f, g, fo, go, nx, ny, nz, sms);
    run<__half, true, false>(f, g, fo, go, nx, ny, nz, sms);
    run<__half, false, true>(f, g, fo, go, nx, ny, nz, sms);
    run<__half, true, true>(f, g, fo, go, nx, ny, nz, sms);
    cudaError_t e = cudaDeviceSynchronize();
    printf("status %s\n", cudaGetErrorString(e));
    cudaFree(f); cudaFree(g); cudaFree(fo); cudaFree(go);
    return e != cudaSuccess;
}
