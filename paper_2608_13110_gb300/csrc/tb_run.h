// Host runtime shared by the C-ABI entry points (api.cu, batch.cu): workspace
// layout of one evaluation and the launch sequence of the sweep.
#pragma once

#include <cstdint>
#include <string>

#include "tb_plan.h"

namespace tb {
namespace rt {

// Record msg as this thread's last error and return code.
int fail(int code, const std::string& msg);

#define TB_CUDA(call)                                                                   \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return ::tb::rt::fail(TB_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

constexpr int64_t DEFAULT_BATCH_ENTRIES = (int64_t)1 << 30;  // 8 GiB of boundaries

// Per-bitstring device bytes of the HBM-pass path (zero for narrow plans).
struct CallLayout {
    int nslots = 0;
    int64_t scale_bytes = 0;     // rescaling slots
    int red_blocks = 0;          // reduction blocks
    int64_t partial_bytes = 0;   // reduction partial sums
    int64_t boundary_bytes = 0;  // the boundary, 8 * 2^h
    int64_t second_bytes = 0;    // open plans out of place: second buffer (join output, late ping-pong), 8 * 2^h
    bool open_in_place = false;  // open plans in place: late crossings over strided rows, and a join
                                 // in row slices through second_bytes of scratch (tensor cores) or,
                                 // when join_slice_rows is 0, in FP32 over the boundary itself
    int64_t join_slice_rows = 0;  // in place: boundary rows per tensor-core join slice
    int64_t per_b = 0;
};

bool small_path(const Plan& P);
// Bytes of one input row (a bitstring, or an open plan's prefix) and amplitudes per row.
inline int64_t in_row(const Plan& P) { return P.open_k ? P.n - P.open_k : P.n; }
inline int64_t amps_per_row(const Plan& P) { return (int64_t)1 << P.open_k; }
CallLayout call_layout(const Plan& P);
int64_t max_batch(const Plan& P, const CallLayout& c);
int num_sms();

// Enqueue the sweep for nb device-resident bitstrings on stream st; the
// plan's tables are at the head of d_ws, the per-bitstring region starts at
// region_off. Returns a tb_status.
// fault: device int that kernels whose bounded waits give up increment (NULL:
// the library-wide word read by tb_device_faults).
int run_device(const Plan& P, const uint8_t* d_bits, int64_t nb, void* d_ws, int64_t ws_bytes,
               int64_t region_off, double* d_out, cudaStream_t st, int* fault = nullptr);

}  // namespace rt
}  // namespace tb
