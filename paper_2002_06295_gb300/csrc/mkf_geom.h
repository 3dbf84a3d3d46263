// mkf_geom.h -- what the kernels see of the context: the device geometry table
// and the device status bits (separate from the host-side context in
// mkf_internal.h, so that a kernel's sources are the kernel file, the device
// math and this header).
#pragma once
#include <stdint.h>

#include "mkf.h"

namespace mkf {

// Device status bits (latched, read and cleared by mkf_sync).
enum : int {
  kStatCapacity = 1,   // a fixed-size device buffer overflowed
  kStatTimeout = 2,    // a bounded wait / iteration limit expired
  kStatBadInput = 4,   // an input index was out of range (skipped)
};

struct LayerDev {
  int kind;
  float pos, lo, hi, x0;
  int nphi, nw, bin_base;
  float phi_scale;   // nphi / (2 pi)
  float w_scale;     // nw / (hi - lo)
  float pad0;        // 11 words: an odd stride keeps lanes reading different layers off one bank
};
static_assert(sizeof(LayerDev) == 44, "LayerDev layout");

struct GeomDev {
  int n_layers;
  float bz;
  float c_kappa;         // -alpha * bz: omega = c_kappa * kappa
  int bins_per_event;
  int n_barrel, n_dpos, n_dneg;
  float r_max;           // outer radius of the tracking volume
  int8_t barrel_order[MKF_MAX_LAYERS];   // barrel ids by increasing r
  int8_t dpos_order[MKF_MAX_LAYERS];     // z > 0 disk ids by increasing z
  int8_t dneg_order[MKF_MAX_LAYERS];     // z < 0 disk ids by increasing |z|
  float barrel_r[MKF_MAX_LAYERS];        // radius of barrel_order[i]
  float dpos_z[MKF_MAX_LAYERS];          // |z| of dpos_order[i]
  float dneg_z[MKF_MAX_LAYERS];          // |z| of dneg_order[i]
  LayerDev L[MKF_MAX_LAYERS];
};
static_assert(sizeof(GeomDev) % 16 == 0, "GeomDev is copied to shared memory in 16-byte words");

}  // namespace mkf
