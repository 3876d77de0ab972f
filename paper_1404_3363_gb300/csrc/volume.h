// The volume handle behind the C ABI (library-internal): host image of the
// prepared volume, its device arrays, transfer function, counters and the
// buffers of the learned initial guess.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <vector>

#include "ivv_device.cuh"
#include "ivv_internal.h"
#include "mlp.cuh"

struct ivv_volume {
  ivv::HostVolume hv;
  int device = 0;
  int num_sms = 1;
  ivv::BlockInfo* d_blocks = nullptr;
  float* d_brk32 = nullptr;
  double* d_brk64 = nullptr;
  float4* d_elem32 = nullptr;
  ivv::Dbl4* d_elem64 = nullptr;
  float4* d_org32 = nullptr;
  float* d_rho32 = nullptr;
  ivv::Dbl4* d_org64 = nullptr;
  // IVV_SCALAR_VONMISES: displacement elements and origins (null otherwise)
  float4* d_disp32 = nullptr;
  float4* d_dorg32 = nullptr;
  ivv::Dbl4* d_disp64 = nullptr;
  ivv::Dbl4* d_dorg64 = nullptr;
  float4* d_face32 = nullptr;
  ivv::Dbl4* d_face64 = nullptr;
  ivv::FaceMeta* d_faces = nullptr;
  ivv::FaceMeta64* d_faces64 = nullptr;
  float* d_tf_r = nullptr;
  float4* d_tf_rgba = nullptr;
  int tf_n = 0;
  std::vector<float> tf_r_host, tf_rgba_host;   // host copy of the TF
  float sigma = 1.f;
  double lo = 0, hi = 1;
  bool tf_set = false;
  ivv::DevStats* d_stats = nullptr;
  int* d_count = nullptr;          // device copy of a point count (point location)
  void* own_ws = nullptr;
  size_t own_ws_bytes = 0;
  float* own_out = nullptr;
  size_t own_out_bytes = 0;
  // ivv_render_to_host_async: two device images used in turn, each copied
  // to the host on copy_stream once its render is done
  float* own_out2[2] = {nullptr, nullptr};
  size_t own_out2_bytes[2] = {0, 0};
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t ev_rendered[2] = {}, ev_copied[2] = {};
  int next_slot = 0;
  cudaStream_t last_stream = nullptr;
  cudaEvent_t ev[IVV_N_STAGES + 1] = {};
  bool timed = false;
  // learned initial guess
  float* d_theta = nullptr;        // [n_blocks][kMlpStride]
  float* d_adam_m = nullptr;
  float* d_adam_v = nullptr;
  __half* d_theta16 = nullptr;
  ivv::MlpNorm* d_norms = nullptr;
  std::vector<ivv::MlpNorm> norms;
  bool guess_ready = false;
  // RF sample buffers (grown on demand)
  void* rf_buf = nullptr;
  size_t rf_bytes = 0;
  // sample lists of the split ODE integration (grown on demand)
  void* ode_buf = nullptr;
  size_t ode_bytes = 0;
  // capacities and iteration caps of the render (ivv_set_limits)
  int lim_frags = ivv::kMaxFrags, lim_pairs = ivv::kMaxPairs, lim_items = ivv::kItemsPerPixel;
  int lim_rk_steps = 200000, lim_newton = 16;
  // overflow and cap counters already reported by ivv_check_frame
  unsigned long long seen_overflow = 0, seen_cap = 0;
};
