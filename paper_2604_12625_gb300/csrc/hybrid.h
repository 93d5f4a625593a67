// Internal types of the hybrid feature map decoder (hybrid.cu).
#pragma once
#include "ndgi_internal.h"

namespace ndgi {

// Device view of one ndgi_hybrid_desc (plus its prepared workspace).
struct DevHybrid {
  int lm_w, lm_h;
  int uv_w, uv_h;
  const uint8_t* uv;
  int vol_w, vol_h, vol_t;
  const uint8_t* vol;
  int ut_w, ut_t;
  const uint8_t* ut;
  int vt_h, vt_t;
  const uint8_t* vt;
  int hidden;
  const float *w1, *b1, *w2, *b2, *w3, *b3;
  int address_mode;
  int bc7;             // F_uv and F3D are BC7 blocks (else four BC4 planes)
  unsigned char* ws;   // FP16/BF16 image and error/debug words, or null (FP32)
};

// One page-decode launch over a table of hybrid models.
struct HybridPagesCtx {
  const DevHybrid* models;   // device array
  int n_models;
  void* phys;
  int64_t phys_w, phys_h;
  int fmt;                   // ndgi_out_format
  int* error_word;           // bit 0 bad request, bit 4 timeout
  const int* debug_word;     // kDbgInjectTimeout
  int border;                // mirrored tile border (texels per edge), 0..8
  int uv_stage;              // some model holds a BC7 F_uv: the launch carries the decoded-footprint buffer
};

}  // namespace ndgi
