// noalloc.cu -- pmmf_apply_noalloc: the matrix-free apply without any device
// allocation, for callers that must not allocate (see include/pmmf.h).
//
// The apply's only scratch is the core slice of the vectors (core_size x nrhs
// doubles) that H and H^-1 read.  Here it lives in one file-scope device array
// of NOALLOC_SCRATCH doubles (8 MiB) that every GPU loading the library keeps
// until the process exits.  The array's name in host code is only a host-side
// stand-in, so its device address is looked up once per device with
// cudaGetSymbolAddress (with that device current) and passed to the kernels.
#include <mutex>
#include <string>

#include "apply.cuh"
#include "common.cuh"

namespace pmmf {
pmmf_status handle_views(const pmmf_handle *f, const ApplyStages **views, HData *H, int64_t *n,
                         bool *inverse_ready, bool *isqrt_ready);
}

namespace {

constexpr int64_t NOALLOC_SCRATCH = int64_t(1) << 20;   // doubles
constexpr int MAX_DEVICES = 64;

static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_SCRATCH];

std::mutex g_scratch_mu;
double *g_scratch_addr[MAX_DEVICES] = {};

// Device address of the scratch array on the current device (set-up on the
// first call per device).
pmmf_status scratch_address(double **out) {
    int dev = 0;
    PMMF_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= MAX_DEVICES) {
        pmmf::set_error("pmmf_apply_noalloc: device ordinal out of range");
        return PMMF_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            pmmf::set_error(std::string("pmmf_apply_noalloc: cudaGetSymbolAddress failed: ") +
                            cudaGetErrorString(e));
            return PMMF_ERR_CUDA;
        }
        g_scratch_addr[dev] = (double *)p;
    }
    *out = g_scratch_addr[dev];
    return PMMF_OK;
}

}  // namespace

using namespace pmmf;

extern "C" pmmf_status pmmf_apply_noalloc(const pmmf_handle *f, int op, const double *x, double *y,
                                          int64_t nrhs, int64_t ld, void *stream) {
    set_error("");
    if (!f || !x || !y) {
        set_error("NULL handle or vector");
        return PMMF_ERR_INVALID_ARG;
    }
    if (nrhs < 1 || ld < nrhs) {
        set_error("need nrhs >= 1 and ld >= nrhs");
        return PMMF_ERR_INVALID_ARG;
    }
    if (op < PMMF_OP_A || op > PMMF_OP_H_INV_SQRT) {
        set_error("unknown op");
        return PMMF_ERR_INVALID_ARG;
    }
    const ApplyStages *views = nullptr;
    HData H;
    int64_t n = 0;
    bool inv_ready = false, isqrt_ready = false;
    PMMF_TRY(handle_views(f, &views, &H, &n, &inv_ready, &isqrt_ready));
    const bool uses_h = op != PMMF_OP_U && op != PMMF_OP_UT;
    const int mode = op == PMMF_OP_A_INV || op == PMMF_OP_H_INV ? 1
                   : op == PMMF_OP_A_INV_SQRT || op == PMMF_OP_H_INV_SQRT ? 2 : 0;
    if (uses_h && H.m * nrhs > NOALLOC_SCRATCH) {
        set_error("pmmf_apply_noalloc: core_size * nrhs = " + std::to_string(H.m * nrhs) +
                  " exceeds the scratch limit of " + std::to_string(NOALLOC_SCRATCH) + " doubles");
        return PMMF_ERR_UNSUPPORTED;
    }
    if (mode == 1 && !inv_ready) {
        set_error("pmmf_apply_noalloc: the core inverse is not formed yet; call pmmf_apply once "
                  "with PMMF_OP_A_INV or PMMF_OP_H_INV first");
        return PMMF_ERR_INVALID_ARG;
    }
    if (mode == 2 && !isqrt_ready) {
        set_error("pmmf_apply_noalloc: the core inverse square root is not formed yet; call "
                  "pmmf_apply once with PMMF_OP_A_INV_SQRT or PMMF_OP_H_INV_SQRT first");
        return PMMF_ERR_INVALID_ARG;
    }
    double *scratch = nullptr;
    PMMF_TRY(scratch_address(&scratch));
    cudaStream_t st = (cudaStream_t)stream;
    if (x != y) PMMF_TRY(copy_block(x, ld, y, ld, n, nrhs, st));
    switch (op) {
    case PMMF_OP_U: return apply_rotations(*views, false, y, ld, nrhs, st);
    case PMMF_OP_UT: return apply_rotations(*views, true, y, ld, nrhs, st);
    case PMMF_OP_H:
    case PMMF_OP_H_INV:
    case PMMF_OP_H_INV_SQRT: return apply_h_scratch(H, mode, y, ld, nrhs, scratch, st);
    default:
        PMMF_TRY(apply_rotations(*views, false, y, ld, nrhs, st));
        PMMF_TRY(apply_h_scratch(H, mode, y, ld, nrhs, scratch, st));
        return apply_rotations(*views, true, y, ld, nrhs, st);
    }
}
