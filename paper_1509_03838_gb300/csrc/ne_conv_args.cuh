// Arguments of the single-job convolution kernels (ne_conv.cu and the
// raw-plane tcgen05 kernels of ne_conv_tcr_w32.cu / ne_conv_tcr_w64.cu),
// and the host interface of the latter.
#pragma once

#include "ne_common.cuh"

namespace ne {

struct ConvArgs {
  const void* x;   // input rows (raw, entangled, or raw to entangle on load)
  int64_t ldx;
  int M;
  int64_t N;
  int64_t Nout;
  int64_t ntiles;
  const int32_t* g;
  int K;
  int Kp;          // K rounded up to CONV_KC
  void* y;         // output rows
  int64_t ldy;
  uint32_t live_mask;  // plain conv: streams to compute
  int l;               // entanglement shift (protected kernel)
  int failed;
  int fail_mode;
  uint32_t* ws;        // protected kernel: per-tile {claim, ready} words
  long long bias;      // MODE_WIDE range shift b (x - b fits 32 bits)
  int kind;            // NE_CONV_LINEAR / NE_CONV_CIRCULAR / NE_CONV_XCORR
  // raw-plane tcgen05 kernels (ne_conv_tcr.cuh)
  int nd;              // byte digits of x - bias
  int hist, ks;        // history samples (K - 1 rounded up to 16), k-steps
  int tcols, tslots;   // tensor-memory columns per stream slot, slots
  int mlev;            // protected: first level of the neighbour's products
                       // in the stream's own levels (l = 8 mlev), 0: apart
  int vec;             // rows of x 16-byte aligned
  unsigned long long corr_mul;  // range-shift correction per unit tap sum
  int lk;              // the large-K form (66 <= K <= 1025)
  const void* btab;    // large K: the taps' B table, tr_table_bytes(K)
                       // bytes, 16-byte aligned (filled by the launch)
  int ytma;            // output rows stored by tensor copies (two tensor
                       // maps passed beside the arguments, rows of even and
                       // of odd index), else by the threads
  int yoff[2];         // per row class: leading outputs of a row before its
                       // first 16-byte boundary (the map starts there)
  int64_t yfull[2];    // per row class: outputs of a row up to the end of
                       // the map's last whole 128-byte piece
  uint32_t wait_limit; // polls before a wait gives up (0: default)
  int stall_role;      // fault injection: 1 loader, 2 MMA issue never run
};

// Geometry of the raw-plane tcgen05 kernels: 128 rows of 32 outputs per
// tile and stream, history of K - 1 <= 64 samples.
constexpr int TR_P = 32;
constexpr int TR_TILE = 128 * TR_P;
constexpr int TR_HMAX = 64;
// The large-K form (66 <= K <= 1025): history up to 1024 samples; its B
// table (tr_table_bytes) lies in global memory.
constexpr int TR_HMAX_L = 1024;
inline size_t tr_table_bytes(int K) {
  const int hist = 16 * ((K - 1 + 15) / 16);
  return (size_t)((TR_P + hist) / 16) * 2048;
}

// Launch the raw-plane kernel for a planned job (ConvArgs fields nd, hist,
// ks, tcols, tslots, vec, corr_mul filled; M, nd within the instantiated
// forms: plain nd 1..4, protected 3 <= M <= 6 and nd 1..2; merged levels
// for M = 4 only); NE_ERR_UNSUPPORTED when the form cannot run here.
int tcr_launch_w32(const ConvArgs& a, bool prot, cudaStream_t s);
int tcr_launch_w64(const ConvArgs& a, bool prot, cudaStream_t s);
// The forms for output rows of a class 8 bytes past a 16-byte boundary
// (a planned by the entry points above, output maps built; tm points to the
// two CUtensorMaps).
int tcr_launch_w32s(const ConvArgs& a, const void* tm, bool prot, cudaStream_t s);
int tcr_launch_w64s(const ConvArgs& a, const void* tm, bool prot, cudaStream_t s);
// The large-K forms (a.lk set, a.btab given).
int tcr_launch_w32l(const ConvArgs& a, const void* tm, bool prot, cudaStream_t s);
int tcr_launch_w64l(const ConvArgs& a, const void* tm, bool prot, cudaStream_t s);
// Host readers of those translation units' device error words.
unsigned tcr_w32_device_error(bool clear);
unsigned tcr_w64_device_error(bool clear);
unsigned tcr_w32s_device_error(bool clear);
unsigned tcr_w64s_device_error(bool clear);
unsigned tcr_w32l_device_error(bool clear);
unsigned tcr_w64l_device_error(bool clear);

}  // namespace ne
