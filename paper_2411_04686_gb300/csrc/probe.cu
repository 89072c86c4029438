// probe.cu -- machine probes behind the roofline denominators that the
// GSE kernels are measured against (gse_probe in include/gse.h).
//
// GB300 is the first GPU in this line whose FP64 rate is far below what a
// memory-bound SpMV needs, so two of the SpMV's floors are not HBM: the FP64
// FMA issue rate (one DFMA per nonzero) and, for scattered columns, the rate
// at which random 8-byte x gathers are served.  These kernels measure both,
// plus the DFMA latency and the rate reached with a given number of dependent
// FMA chains per SM (how much independent work an SpMV must keep in flight).
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/gse.h"

namespace {

// DFMA throughput: every thread runs C independent chains of n dependent
// FMAs.  The values stay finite (|a| < 1 contracts towards b / (1 - a)).
template <int C>
__global__ void k_dfma_rate(int n, double a, double b, double* sink) {
    double v[C];
#pragma unroll
    for (int c = 0; c < C; c++) v[c] = (double)(threadIdx.x + c);
    for (int i = 0; i < n; i++) {
#pragma unroll
        for (int c = 0; c < C; c++) v[c] = fma(v[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < C; c++) s += v[c];
    if (s == 12345.678) sink[0] = s;   // never true; keeps the chains live
}

// DFMA latency: one thread, one dependent chain, timed with the SM clock.
__global__ void k_dfma_latency(int n, double a, double b, double* out) {
    double v = (double)threadIdx.x;
    const long long t0 = clock64();
    for (int i = 0; i < n; i++) v = fma(v, a, b);
    const long long t1 = clock64();
    out[0] = (double)(t1 - t0) / n;
    out[1] = v;
}

// Random 8-byte gathers: each thread issues G independent loads per round
// from a table of `words` doubles (indices from a 32-bit mix of the thread,
// round and slot; the table is a power of two).  MODE 0: through L1
// (ld.global.nc); MODE 1: L2 only (ld.global.cg).
__device__ __forceinline__ uint32_t mix32(uint32_t v) {
    v ^= v >> 16;
    v *= 0x7feb352dU;
    v ^= v >> 15;
    v *= 0x846ca68bU;
    v ^= v >> 16;
    return v;
}

template <int G, int MODE>
__global__ void k_gather_rate(const double* __restrict__ t, uint32_t mask, int rounds, double* sink) {
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    double s = 0.0;
    for (int r = 0; r < rounds; r++) {
        double v[G];
#pragma unroll
        for (int g = 0; g < G; g++) {
            const uint32_t i = mix32(tid * 0x9E3779B9u + (uint32_t)(r * G + g) * 0x85EBCA6Bu) & mask;
            if constexpr (MODE == 0) v[g] = __ldg(t + i);
            else v[g] = __ldcg(t + i);
        }
#pragma unroll
        for (int g = 0; g < G; g++) s += v[g];
    }
    if (s == 12345.678) sink[0] = s;
}

float time_ms(cudaStream_t s, void (*launch)(cudaStream_t, void*), void* arg, int reps) {
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    launch(s, arg);   // warm
    cudaEventRecord(e0, s);
    for (int i = 0; i < reps; i++) launch(s, arg);
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return ms / reps;
}

struct RateArg {
    int blocks, threads, n, chains;
    double* sink;
};

void launch_rate(cudaStream_t s, void* p) {
    const RateArg* a = (const RateArg*)p;
    switch (a->chains) {
        case 1: k_dfma_rate<1><<<a->blocks, a->threads, 0, s>>>(a->n, 0.999, 0.5, a->sink); break;
        case 2: k_dfma_rate<2><<<a->blocks, a->threads, 0, s>>>(a->n, 0.999, 0.5, a->sink); break;
        case 4: k_dfma_rate<4><<<a->blocks, a->threads, 0, s>>>(a->n, 0.999, 0.5, a->sink); break;
        default: k_dfma_rate<8><<<a->blocks, a->threads, 0, s>>>(a->n, 0.999, 0.5, a->sink); break;
    }
}

struct GatherArg {
    const double* t;
    uint32_t mask;
    int blocks, threads, rounds, mode;
    double* sink;
};

void launch_gather(cudaStream_t s, void* p) {
    const GatherArg* a = (const GatherArg*)p;
    if (a->mode == 0) k_gather_rate<8, 0><<<a->blocks, a->threads, 0, s>>>(a->t, a->mask, a->rounds, a->sink);
    else k_gather_rate<8, 1><<<a->blocks, a->threads, 0, s>>>(a->t, a->mask, a->rounds, a->sink);
}

}  // namespace

extern "C" int gse_probe(int which, int64_t param, const double* table, double* out, void* stream) {
    if (!out) return GSE_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 1;
    if (cudaGetDevice(&dev) != cudaSuccess) return GSE_ERR_CUDA;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    double* sink = nullptr;
    if (cudaMallocAsync(&sink, 2 * sizeof(double), s) != cudaSuccess) {
        cudaGetLastError();
        return GSE_ERR_OOM;
    }
    int rc = GSE_OK;
    if (which == GSE_PROBE_DFMA_RATE || which == GSE_PROBE_DFMA_CHAINS) {
        // RATE: full occupancy, 8 chains per thread.  CHAINS: `param` warps per
        // SM with one chain per thread (the dependent-chain regime of an SpMV row).
        RateArg a;
        a.sink = sink;
        a.n = 4096;
        if (which == GSE_PROBE_DFMA_RATE) {
            a.threads = 256;
            a.blocks = sms * 8;
            a.chains = 8;
        } else {
            if (param < 1 || param > 64) { cudaFreeAsync(sink, s); return GSE_ERR_INVALID; }
            a.threads = 32;
            a.blocks = sms * (int)param;
            a.chains = 1;
        }
        const float ms = time_ms(s, launch_rate, &a, 5);
        out[0] = (double)a.blocks * a.threads * a.chains * a.n / (ms * 1e-3);   // FMA / s
        out[1] = ms;
    } else if (which == GSE_PROBE_DFMA_LATENCY) {
        k_dfma_latency<<<1, 1, 0, s>>>(4096, 0.999, 0.5, sink);
        k_dfma_latency<<<1, 1, 0, s>>>(4096, 0.999, 0.5, sink);
        double h[2] = {0, 0};
        cudaMemcpyAsync(h, sink, sizeof(h), cudaMemcpyDeviceToHost, s);
        cudaStreamSynchronize(s);
        out[0] = h[0];   // SM cycles per dependent DFMA
        out[1] = 0.0;
    } else if (which == GSE_PROBE_GATHER_L1 || which == GSE_PROBE_GATHER_L2) {
        // param: table size in doubles, a power of two; the caller owns the table
        if (!table || param < 1024 || (param & (param - 1)) != 0 || param > ((int64_t)1 << 32)) {
            cudaFreeAsync(sink, s);
            return GSE_ERR_INVALID;
        }
        GatherArg a;
        a.t = table;
        a.mask = (uint32_t)(param - 1);
        a.threads = 256;
        a.blocks = sms * 8;
        a.rounds = 64;
        a.mode = which == GSE_PROBE_GATHER_L1 ? 0 : 1;
        a.sink = sink;
        const float ms = time_ms(s, launch_gather, &a, 5);
        out[0] = (double)a.blocks * a.threads * a.rounds * 8 / (ms * 1e-3);      // gathers / s
        out[1] = ms;
    } else {
        rc = GSE_ERR_INVALID;
    }
    cudaFreeAsync(sink, s);
    if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess) rc = GSE_ERR_CUDA;
    return rc;
}
