// Dumps cuRAND device-API philox4_32_10 blocks: state from curand_init(seed,
// subsequence = path0 + i, offset = 0), then curand4() n_calls times.  Used by
// the GPU test that checks the library's counter layout against cuRAND.
#include <cstdio>
#include <cstdlib>
#include <curand_kernel.h>

__global__ void dump(unsigned long long seed, unsigned long long path0, int n_paths, int n_calls,
                     uint4 *out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_paths) return;
    curandStatePhilox4_32_10_t st;
    curand_init(seed, path0 + (unsigned long long)i, 0, &st);
    for (int c = 0; c < n_calls; ++c) out[(size_t)i * n_calls + c] = curand4(&st);
}

int main(int argc, char **argv) {
    if (argc != 5) return 2;
    unsigned long long seed = strtoull(argv[1], 0, 0), path0 = strtoull(argv[2], 0, 0);
    int n_paths = atoi(argv[3]), n_calls = atoi(argv[4]);
    if (n_paths < 1 || n_calls < 1 || n_paths > 4096 || n_calls > 64) return 2;
    size_t n = (size_t)n_paths * n_calls;
    uint4 *d = nullptr;
    if (cudaMalloc(&d, n * sizeof(uint4)) != cudaSuccess) return 3;
    dump<<<(n_paths + 127) / 128, 128>>>(seed, path0, n_paths, n_calls, d);
    uint4 *h = (uint4 *)malloc(n * sizeof(uint4));
    if (cudaMemcpy(h, d, n * sizeof(uint4), cudaMemcpyDeviceToHost) != cudaSuccess) return 4;
    fwrite(h, sizeof(uint4), n, stdout);
    cudaFree(d);
    free(h);
    return 0;
}
