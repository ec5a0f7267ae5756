// Distributed-shared-memory (DSMEM) exchange rate on sm_103a, measured the
// way a frame split over a thread-block cluster would use it: every CTA of a
// cluster holds part of a frame in registers and, per exchange, writes a
// fixed number of bytes into the shared memory of the other CTAs of its
// cluster, then the cluster synchronises once.  Variants:
//   local   : the same stores into the CTA's own shared memory (baseline)
//   remote  : 16-byte st.shared::cluster.v4 stores to the peer CTAs (mapa)
//   remote8 : 8-byte st.shared::cluster.v2 stores
//   bulk    : one bulk copy (cp.async.bulk shared::cta -> shared::cluster)
//             per peer from a local send buffer, completing on the receiver's
//             mbarrier (the copy engine moves the bytes, not the threads)
//   l2      : the same bytes stored to and re-read from a per-CTA global slab
//             (what the 256^2 line-pass kernel does between passes)
// Each variant runs `reps` exchanges of `bytes_per_cta` in a grid of as many
// clusters of cs CTAs x 512 threads as can be resident at once (all 152 SMs
// for cs = 1, 2; fewer for 4 and 8, whose clusters must fit a GPC); the rate
// is reported per SM and for the whole GPU.  One cluster barrier closes every
// exchange (two for the remote variants: buffers free, data arrived), and
// the barrier cost is measured alone with zero bytes.
//
// Build and run (one GPU):
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -std=c++17 \
//        paper_1602_01448_gb300/microbench/dsmem_rate.cu -o dsmem_rate && ./dsmem_rate
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#define CK(x)                                                                           \
    do {                                                                                \
        cudaError_t e_ = (x);                                                           \
        if (e_ != cudaSuccess) {                                                        \
            fprintf(stderr, "%s:%d %s: %s\n", __FILE__, __LINE__, #x, cudaGetErrorString(e_)); \
            return 1;                                                                   \
        }                                                                               \
    } while (0)

constexpr int NT = 512;
constexpr int BUF_BYTES = 128 * 1024;   // receive buffer per CTA
constexpr int SEND_BYTES = 64 * 1024;   // send buffer of the bulk variant
constexpr unsigned kPolls = 1u << 24;   // bound of every mbarrier wait

__device__ __forceinline__ unsigned cluster_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ unsigned cluster_size() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ unsigned map_rank(unsigned saddr, unsigned rank) {
    unsigned r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
    return r;
}
__device__ __forceinline__ void st_cluster_v4(unsigned addr, float4 v) {
    asm volatile("st.shared::cluster.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "f"(v.x), "f"(v.y), "f"(v.z),
                 "f"(v.w)
                 : "memory");
}
__device__ __forceinline__ void st_cluster_v2(unsigned addr, float2 v) {
    asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(addr), "f"(v.x), "f"(v.y) : "memory");
}

__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect(unsigned bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// Bounded wait (acquire at cluster scope: the bytes came from peers' copies).
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity) {
    for (unsigned it = 0; it < kPolls; ++it) {
        unsigned ok;
        asm volatile("{\n\t.reg .pred p;\n\t"
                     "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
        if (ok) return true;
    }
    return false;
}
__device__ __forceinline__ void bulk_s2cluster(unsigned dst_cluster, unsigned src_cta, unsigned bytes,
                                               unsigned bar_cluster) {
    asm volatile("cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(dst_cluster), "r"(src_cta), "r"(bytes), "r"(bar_cluster) : "memory");
}

enum Variant { LOCAL = 0, REMOTE = 1, REMOTE8 = 2, L2SLAB = 3, BULK = 4 };

// Bulk variant: per exchange each CTA sends bytes_per_cta / (cs - 1) to every
// peer, one bulk copy each, into the peer's receive buffer at the slot of
// the sender; the receiver's mbarrier counts the bytes.
__global__ void __launch_bounds__(NT, 1) bulk_kernel(int reps, int bytes_per_cta, int* timeouts, float* sink) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) unsigned long long rbar;
    const unsigned rank = cluster_rank(), cs = cluster_size();
    const int tid = threadIdx.x;
    const unsigned recv = (unsigned)__cvta_generic_to_shared(smem);
    const unsigned send = recv + BUF_BYTES;
    const unsigned bar = (unsigned)__cvta_generic_to_shared(&rbar);
    const unsigned chunk = cs > 1 ? (unsigned)(bytes_per_cta / (cs - 1)) & ~15u : 0u;
    for (int k = tid; k < SEND_BYTES / 4; k += NT) reinterpret_cast<float*>(smem + BUF_BYTES)[k] = (float)(k + rank);
    if (tid == 0) mbar_init(bar, 1);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // send buffer -> copy engine
    cluster_sync();
    unsigned parity = 0;
    float acc = 0.f;
    bool ok = true;
    for (int r = 0; r < reps; ++r) {
        if (tid == 0) mbar_expect(bar, chunk * (cs - 1));
        cluster_sync();                                          // receivers armed, buffers free
        if (tid > 0 && (unsigned)tid < cs && chunk > 0) {          // one thread per peer
            const unsigned peer = (rank + (unsigned)tid) % cs;
            const unsigned slot = (cs + rank - peer - 1) % cs;    // sender's slot at the peer: 0 .. cs-2
            bulk_s2cluster(map_rank(recv + slot * chunk, peer), send, chunk, map_rank(bar, peer));
        }
        if (tid == 0) ok = ok && mbar_wait(bar, parity);
        parity ^= 1u;
        __syncthreads();
        acc += reinterpret_cast<const float*>(smem)[tid];
    }
    if (tid == 0 && !ok) atomicAdd(timeouts, 1);
    cluster_sync();                                              // all copies into every CTA landed
    if (acc == 12345.f) sink[0] = acc;
}

// bytes_per_cta: bytes each CTA sends per exchange (<= BUF_BYTES, multiple
// of 16 * NT).  The sent values depend on the registers so that the stores
// cannot be removed; `sink` keeps a checksum of what was received.
template <int VAR>
__global__ void __launch_bounds__(NT, 1) exchange_kernel(int reps, int bytes_per_cta, float4* slab, float* sink) {
    extern __shared__ __align__(128) unsigned char smem[];
    const unsigned rank = cluster_rank(), cs = cluster_size();
    const int tid = threadIdx.x;
    const int per_thread = bytes_per_cta / (16 * NT);   // 16-byte units per thread
    float4 v = make_float4(tid, rank, 1.f, 2.f);
    const unsigned base = (unsigned)__cvta_generic_to_shared(smem);
    float4* slab_cta = slab + (size_t)blockIdx.x * (BUF_BYTES / 16);
    float acc = 0.f;
    for (int r = 0; r < reps; ++r) {
        if (VAR == REMOTE || VAR == REMOTE8) cluster_sync();   // peers' buffers are free
        for (int u = 0; u < per_thread; ++u) {
            const int slot = u * NT + tid;                          // 16-byte slot in the buffer
            const unsigned peer = (rank + 1 + (unsigned)(slot % (cs > 1 ? cs - 1 : 1))) % cs;
            if (VAR == LOCAL) {
                reinterpret_cast<float4*>(smem)[slot] = v;
            } else if (VAR == REMOTE) {
                st_cluster_v4(map_rank(base + 16u * slot, peer), v);
            } else if (VAR == REMOTE8) {
                const unsigned a = map_rank(base + 16u * slot, peer);
                st_cluster_v2(a, make_float2(v.x, v.y));
                st_cluster_v2(a + 8, make_float2(v.z, v.w));
            } else {
                slab_cta[slot] = v;
            }
            v.x += 1.f;
        }
        if (VAR == L2SLAB) {
            __syncthreads();
            for (int u = 0; u < per_thread; ++u) {
                const float4 t = __ldcg(slab_cta + (u * NT + (tid ^ 32)));
                acc += t.x;
            }
        } else {
            if (VAR == LOCAL) __syncthreads();
            else cluster_sync();                                    // data arrived
            for (int u = 0; u < per_thread; ++u) acc += reinterpret_cast<float4*>(smem)[u * NT + (tid ^ 32)].x;
        }
    }
    if (VAR == REMOTE || VAR == REMOTE8) cluster_sync();           // no CTA exits while peers may write
    if (acc == 12345.f) sink[0] = acc;
}

template <class K, class... Args>
static int run_kernel(const char* name, K k, int smem, int cs, int bytes, int reps, int sms, Args... args) {
    CK(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    CK(cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((sms / cs) * cs);
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nclusters = 0;
    CK(cudaOccupancyMaxActiveClusters(&nclusters, k, &cfg));
    if (nclusters < 1) {
        printf("%-8s cs=%d: no cluster can be resident, skipped\n", name, cs);
        return 0;
    }
    if (nclusters * cs < (int)cfg.gridDim.x) cfg.gridDim = dim3(nclusters * cs);   // one wave
    const int grid = (int)cfg.gridDim.x;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    CK(cudaLaunchKernelEx(&cfg, k, 2, bytes, args...));   // warm-up
    CK(cudaEventRecord(e0));
    CK(cudaLaunchKernelEx(&cfg, k, reps, bytes, args...));
    CK(cudaEventRecord(e1));
    CK(cudaEventSynchronize(e1));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    const double per_ex_us = 1e3 * ms / reps;
    const double gbs_sm = bytes > 0 ? (double)bytes / (per_ex_us * 1e-6) / 1e9 : 0.0;
    printf("%-8s cs=%d bytes/CTA/exchange=%6d: %8.3f us per exchange, %8.1f GB/s per SM, %8.1f GB/s on %d SMs\n",
           name, cs, bytes, per_ex_us, gbs_sm, gbs_sm * grid, grid);
    CK(cudaEventDestroy(e0));
    CK(cudaEventDestroy(e1));
    return 0;
}

template <int VAR>
static int run(const char* name, int cs, int bytes, int reps, float4* slab, float* sink, int sms) {
    return run_kernel(name, exchange_kernel<VAR>, BUF_BYTES, cs, bytes, reps, sms, slab, sink);
}

int main() {
    int dev = 0, sms = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    float4* slab = nullptr;
    float* sink = nullptr;
    CK(cudaMalloc(&slab, (size_t)sms * BUF_BYTES));
    CK(cudaMalloc(&sink, sizeof(float)));
    const int reps = 2000;
    const int sizes[] = {0, 8192 * 4, 96 * 1024, 128 * 1024};
    int* timeouts = nullptr;
    CK(cudaMalloc(&timeouts, sizeof(int)));
    CK(cudaMemset(timeouts, 0, sizeof(int)));
    for (int cs : {2, 4, 8}) {
        for (int b : sizes) {
            if (run<REMOTE>("remote", cs, b, reps, slab, sink, sms)) return 1;
        }
        if (run<REMOTE8>("remote8", cs, 96 * 1024, reps, slab, sink, sms)) return 1;
        for (int b : {32768, 96 * 1024, 128 * 1024}) {
            const int bb = b / (cs - 1) > SEND_BYTES ? SEND_BYTES * (cs - 1) : b;
            if (run_kernel("bulk", bulk_kernel, BUF_BYTES + SEND_BYTES, cs, bb, reps, sms, timeouts, sink)) return 1;
        }
    }
    int to = 0;
    CK(cudaMemcpy(&to, timeouts, sizeof(int), cudaMemcpyDeviceToHost));
    printf("bulk waits that gave up: %d\n", to);
    CK(cudaFree(timeouts));
    for (int b : sizes) {
        if (run<LOCAL>("local", 1, b, reps, slab, sink, sms)) return 1;
        if (run<L2SLAB>("l2slab", 1, b, reps, slab, sink, sms)) return 1;
    }
    CK(cudaFree(slab));
    CK(cudaFree(sink));
    return 0;
}
