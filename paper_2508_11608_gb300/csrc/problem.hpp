// The problem handle shared by the C ABI (capi.cu) and the server (server.cu).
#pragma once

#include <memory>

#include "../../include/cutmg.h"
#include "engine_api.hpp"
#include "setup.hpp"

struct cf_problem {
  cutmg::Hierarchy H;
  std::unique_ptr<cutmg::EngineBase> eng;
  int precision = CF_FP64;
  int device = 0;
};

extern "C" {
// host phase of cf_setup (hierarchy only), device phase (engine + upload)
cf_status cutmg_build_host(const cf_mesh* mesh, const cf_levelset* ls, int degree, const cf_params* params,
                           cf_problem** out);
cf_status cutmg_attach_device(cf_problem* pb, cudaStream_t stream);
// device bytes the engine of a host-built problem will allocate
size_t cutmg_estimate_device_bytes(const cf_problem* pb);
// the same from a hierarchy, also one built with SetupParams::dry (sizes only)
size_t cutmg_estimate_hierarchy_bytes(const cutmg::Hierarchy& H);
}
cf_status cutmg_set_error(cf_status s, const char* msg);
