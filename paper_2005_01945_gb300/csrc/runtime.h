// runtime.h -- host-side context shared by the C-ABI translation units.
#pragma once
#include <mutex>
#include <string>

#include <nvtx3/nvToolsExt.h>

#include "common.cuh"

namespace tgb {
struct CircuitCache;
struct Server;
}  // namespace tgb

struct tfhe_ctx {
    int device = 0;
    tfhe_params prm{};
    int num_sms = 0;
    int br_grid = 0;                 // persistent blind-rotation grid
    uint2 *twb = nullptr;            // stage-B twiddles
    uint32_t *bk_ntt = nullptr;      // bootstrapping key, NTT domain
    uint4 *ksk = nullptr;            // key-switching key, padded rows
    uint32_t *status = nullptr;      // device status word
    int32_t *big = nullptr;          // LWE_N scratch between the two stages
    size_t big_rows = 0;
    bool keys_loaded = false;
    tgb::DevKeys keys{};
    std::string err;                 // last failure message (guarded by err_mu: the
    mutable std::mutex err_mu;       // serving calls fail from several threads)
    uint64_t launches = 0;           // kernels issued (graph nodes count per replay)
    size_t test_free_hbm = 0;        // test hook: serving takes this as the free HBM
    tgb::CircuitCache *circuits = nullptr;
    tgb::Server *server = nullptr;
};

namespace tgb {

struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess)
            prev = -1;
        ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard()
    {
        if (prev >= 0)
            cudaSetDevice(prev);
    }
};

// A named range on the host timeline of profilers (NVTX; costs a pointer
// check when no profiler is attached): one per phase a call enqueues.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

int fail(tfhe_ctx *ctx, int code, const char *fmt, ...);
int cuda_fail(tfhe_ctx *ctx, cudaError_t e, const char *where);
bool params_supported(const tfhe_params *p);
int ensure_big(tfhe_ctx *ctx, size_t rows);
int run_bootstrap(tfhe_ctx *ctx, const uint8_t *ops, const int32_t *a, const int32_t *idx_a,
                  long rows_a, const int32_t *b, const int32_t *idx_b, long rows_b, int32_t *out,
                  const int32_t *idx_out, long rows_out, long count, uint32_t mu,
                  cudaStream_t stream);

cudaError_t launch_blind_rotate(const DevKeys &keys, const uint8_t *ops, const int32_t *in_a,
                                const int32_t *idx_a, long rows_a, const int32_t *in_b,
                                const int32_t *idx_b, long rows_b, int32_t *big, long count,
                                uint32_t mu, uint32_t *status, int grid, cudaStream_t stream,
                                const int32_t *in_c = nullptr, const int32_t *idx_c = nullptr,
                                long rows_c = 0);
cudaError_t launch_keyswitch(const uint4 *ksk, const int32_t *big, int32_t *out,
                             const int32_t *idx_out, long rows_out, long count, int n,
                             int num_sms, uint32_t *status, cudaStream_t stream,
                             const DevKeys *choice = nullptr);

int keyswitch_kernels(long count, int num_sms, const DevKeys *choice = nullptr);
void keyswitch_force_chunks(int chunks);

void release_circuits(tfhe_ctx *ctx);
void invalidate_graphs(tfhe_ctx *ctx);
void release_serving(tfhe_ctx *ctx);

}  // namespace tgb
