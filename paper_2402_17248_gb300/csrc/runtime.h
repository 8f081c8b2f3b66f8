// Host runtime shared by the C-ABI translation units: error reporting,
// per-device context, per-(device, stream) scratch workspaces, reference
// particle tracking and linear element matrices in FP64.
#pragma once
#include <array>
#include <cstdint>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "internal.h"

namespace bl {

// ---- errors ----
bl_status set_error(bl_status st, const std::string &msg);
bl_status cuda_error(cudaError_t e, const char *what);

#define BL_CUDA(expr)                                      \
  do {                                                     \
    cudaError_t _e = (expr);                               \
    if (_e != cudaSuccess) return ::bl::cuda_error(_e, #expr); \
  } while (0)

#define BL_CHECK(cond, msg)                                              \
  do {                                                                   \
    if (!(cond)) return ::bl::set_error(BL_ERR_INVALID_ARG, (msg));      \
  } while (0)

#define BL_TRY(expr)                       \
  do {                                     \
    bl_status _s = (expr);                 \
    if (_s != BL_OK) return _s;            \
  } while (0)

// ---- device context ----
struct DevCtx {
  int device = -1;
  int num_sms = 0;
  bool arch_ok = false;
  unsigned *err_word = nullptr;  // device word for BL_DEVERR_* flags
  bool mlp_configured = false;
  bool mlp_vjp_configured = false;
  bool wide_configured = false;
  bool train_tc_configured = false;
  // bl_track_host pipeline: two compute streams, one stream per copy
  // direction and the events that order them (created on first use)
  cudaStream_t hp_comp[2] = {nullptr, nullptr};
  cudaStream_t hp_h2d = nullptr, hp_d2h = nullptr;
  // events: 4 per chunk buffer for each of copy-in, tracked, copy-out, one
  // start and four joins (indices fixed in bl_track_host)
  static constexpr int HOST_EVENTS = 17;
  cudaEvent_t hp_ev[HOST_EVENTS] = {};
};
// Context of the current device; checks the architecture (sm_103) once.
bl_status current_ctx(DevCtx **out);

// ---- workspaces ----
enum WsSlot {
  WS_PARTIALS = 0, WS_MOMENTS, WS_NONFINITE, WS_TABLES, WS_MATS, WS_CENTERS, WS_LAMBDA,
  WS_CKPT, WS_CROSS, WS_TRAIN, WS_LOSS, WS_WIDE0, WS_WIDE1, WS_FALLBACK, WS_TRAIN_SCRATCH,
  WS_HOST_BUF, WS_HOST_RED, WS_WIDE_TRAIN, WS_TRAIN_ACC, WS_COUNT
};
struct Workspace {
  void *ptr[WS_COUNT] = {};
  size_t bytes[WS_COUNT] = {};
};
// Grow-only device buffer `slot` of the (device, stream) workspace.
bl_status ws_get(cudaStream_t st, WsSlot slot, size_t bytes, void **out);

// ---- physics (FP64, host) ----
struct Consts {
  static constexpr double C = 299792458.0;
  static constexpr double E = 1.602176634e-19;
  static constexpr double EPS0 = 8.8541878128e-12;
  static constexpr double ME = 9.1093837015e-31;
  static constexpr double MEC2_EV = 0.51099895000e6;
};

using Mat6 = std::array<double, 36>;
Mat6 mat_identity();
Mat6 mat_mul(const Mat6 &A, const Mat6 &B);  // A * B
Mat6 mat_transpose(const Mat6 &A);
Mat6 element_matrix(const bl_element &e, double k, double bg);
Mat6 element_dmatrix_dk(const bl_element &e, double k, double bg);  // quads only

// On-axis FP64 reference through one stage with the RK4 of the pusher.
// Fills the constants and, if requested, the per-(step, RK4 stage) table in
// the FP32 or FP64 layout documented in pusher.cu.
struct StageTrack {
  StageConsts c;
  std::vector<float> table32;
  std::vector<double> table64;
};
bl_status stage_track(const bl_element &e, double gamma_in, int want_table_dtype,
                      StageTrack *out);

bool bunch_dims_ok(const bl_bunch *b, std::string *why);

template <typename T> Soa<T> soa_of(const bl_bunch *b) {
  Soa<T> s;
  s.c[0] = static_cast<T *>(b->x);
  s.c[1] = static_cast<T *>(b->px);
  s.c[2] = static_cast<T *>(b->y);
  s.c[3] = static_cast<T *>(b->py);
  s.c[4] = static_cast<T *>(b->t);
  s.c[5] = static_cast<T *>(b->pt);
  return s;
}

// Moments of a bunch into a device buffer (n_bunch x 28 doubles) with the
// streaming kernels; nonfinite counter optional (device).
bl_status moments_device(const bl_bunch *b, double *out_dev, unsigned long long *nonfinite,
                         cudaStream_t st);

// Build (or reuse) the lattice's device plan for a reference energy, dtype and
// bunch count. Caller holds the lattice mutex.
bl_status build_plan(bl_lattice_s *L, double gamma_in, int dtype, int n_bunch, cudaStream_t st);

// 28-vector (N, means, central moments) propagated through a linear map.
void propagate_moments(const Mat6 &M, const double *in28, double *out28);

}  // namespace bl

struct bl_surrogate_s {
  int device = -1;
  float *params = nullptr;  // flat FP32 masters (MLP_NPARAM)
  float *m = nullptr, *v = nullptr;
  uint8_t *img = nullptr;   // BF16 UMMA image
  float *bias = nullptr;    // FP32 bias block
  float *wt = nullptr, *wn = nullptr;  // BF16-rounded FP32 copies
  bl::MlpNorm nrm{};
  double mu_in[6], sd_in[6], mu_out[6], sd_out[6];
  int step = 0;
  bool has_domain = false;      // training-input box set (bl_surrogate_set_domain)
  float dom_lo[6], dom_hi[6];
};

struct bl_wide_mlp_s {
  int device = -1;
  bl::WideNet net;
  float *G = nullptr, *M = nullptr, *V = nullptr;  // flat gradient and Adam moments
  int step = 0;
};

struct bl_lattice_s {
  std::vector<bl_element> els;
  std::vector<std::vector<double>> pbk;  // per-element copy of per_bunch_k
  int n_bunch_k = 0;
  int n_quads = 0;
  // groups: maximal runs of linear elements (segments) and single stages
  struct Group {
    bool stage;
    int first, last;  // element indices, inclusive
  };
  std::vector<Group> groups;
  // cached device plan
  std::mutex mu;
  struct Plan {
    bool valid = false;
    double gamma_in = 0;
    int dtype = -1, n_bunch = 0, device = -1;
    std::vector<bl::StageTrack> stages;          // per group (stage groups only)
    std::vector<std::vector<bl::Mat6>> seg_mats;  // per group: per-bunch segment matrix
    std::vector<std::vector<std::vector<bl::Mat6>>> el_mats;  // per group, element, bunch
    std::vector<size_t> table_off, mat_off;      // byte offsets into device buffers
    void *d_tables = nullptr, *d_mats = nullptr;
    size_t tables_bytes = 0, mats_bytes = 0;
    double gamma_out = 0;
  } plan;
  ~bl_lattice_s();
};
