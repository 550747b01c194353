// Throughput of shared-memory atomics: local vs distributed (cluster), int/f32/f64, spread vs hot.
#include <cooperative_groups.h>
#include <cstdio>
#include <cuda_runtime.h>
namespace cg = cooperative_groups;

constexpr int NT = 1024;
constexpr int SLOTS = 4096;

template <typename T, int MODE>  // MODE 0: local spread, 1: local hot(32 addr), 2: remote spread, 3: remote hot
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(NT) kprobe(int iters, void *sinkv) {
    __shared__ T tab[SLOTS];
    cg::cluster_group cl = cg::this_cluster();
    for (int i = threadIdx.x; i < SLOTS; i += NT) tab[i] = T(0);
    cl.sync();
    T *dst = tab;
    if (MODE >= 2) dst = cl.map_shared_rank(tab, (int)cl.block_rank() ^ 1);
    unsigned x = threadIdx.x * 2654435761u + blockIdx.x;
    for (int it = 0; it < iters; ++it) {
        x = x * 1664525u + 1013904223u;
        int slot = (MODE == 1 || MODE == 3) ? (x >> 27) : (x >> 20) & (SLOTS - 1);
        atomicAdd(dst + slot, T(1));
    }
    cl.sync();
    if (threadIdx.x == 0) ((decltype(&tab[0]))sinkv)[blockIdx.x] = tab[0];
}

template <int MODE>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(NT) kcas_f64(int iters, void *sinkv) {
    __shared__ double tab[SLOTS];
    cg::cluster_group cl = cg::this_cluster();
    for (int i = threadIdx.x; i < SLOTS; i += NT) tab[i] = 0.0;
    cl.sync();
    unsigned x = threadIdx.x * 2654435761u + blockIdx.x;
    for (int it = 0; it < iters; ++it) {
        x = x * 1664525u + 1013904223u;
        int slot = (MODE == 1) ? (x >> 27) : (x >> 20) & (SLOTS - 1);
        unsigned long long *p = (unsigned long long *)(tab + slot);
        unsigned long long old = *p, assumed;
        do {
            assumed = old;
            old = atomicCAS(p, assumed, __double_as_longlong(__longlong_as_double(assumed) + 1.0));
        } while (assumed != old);
    }
    cl.sync();
    if (threadIdx.x == 0) ((decltype(&tab[0]))sinkv)[blockIdx.x] = tab[0];
}

template <typename K>
float timeit(K k, int grid, int iters, void *sink) {
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    k<<<grid, NT>>>(iters, sink);
    cudaEventRecord(a);
    k<<<grid, NT>>>(iters, sink);
    cudaEventRecord(b);
    cudaEventSynchronize(b);
    float ms;
    cudaEventElapsedTime(&ms, a, b);
    return ms;
}

int main() {
    int sms;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
    int grid = sms * 2;  // 2 blocks/SM (1024 thr, 64 KB) -> full occupancy
    void *sink;
    cudaMalloc(&sink, 1 << 20);
    const int iters = 2000;
    double ops = (double)grid * NT * iters;
#define RUN(T, M, name)                                                                         \
    {                                                                                           \
        float ms = timeit(kprobe<T, M>, grid, iters, sink);                                     \
        printf("%-28s %8.3f ms  %8.1f Gop/s  %6.2f op/clk/SM\n", name, ms, ops / ms / 1e6,   \
               ops / (ms * 1e-3) / sms / 1.9e9);                                                \
    }
    RUN(int, 0, "int local spread");
    RUN(int, 1, "int local hot32");
    RUN(int, 2, "int remote spread");
    RUN(int, 3, "int remote hot32");
    RUN(float, 0, "f32 local spread");
    RUN(float, 1, "f32 local hot32");
    RUN(float, 2, "f32 remote spread");
    RUN(float, 3, "f32 remote hot32");
    RUN(double, 0, "f64 local spread");
    RUN(double, 1, "f64 local hot32");
    RUN(double, 2, "f64 remote spread");
    RUN(double, 3, "f64 remote hot32");
    {
        float ms = timeit(kcas_f64<0>, grid, iters, sink);
        printf("%-28s %8.3f ms  %8.1f Gop/s\n", "f64 CAS-loop local spread", ms, ops / ms / 1e6);
        ms = timeit(kcas_f64<1>, grid, iters, sink);
        printf("%-28s %8.3f ms  %8.1f Gop/s\n", "f64 CAS-loop local hot32", ms, ops / ms / 1e6);
    }
    cudaError_t e = cudaDeviceSynchronize();
    printf("status %s\n", cudaGetErrorString(e));
    return e == cudaSuccess ? 0 : 1;
}
