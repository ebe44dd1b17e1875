// Host-side construction and validation of the launch parameters (pgk::Params)
// from the public configuration, camera and radiance-field structs.
#pragma once

#include <string>

#include "../../include/pg.h"
#include "pg_device.cuh"

namespace pgk {

bool aligned16(const void* p);

// Validates a configuration; on failure returns PG_ERR_ARG and a reason.
pg_status check_config(const pg_config* c, std::string& why);

// The configuration part of the launch parameters (sizes, thresholds, the
// re-initialised guide, the Philox key and the rule of Z's corner integrals).
void config_params(const pg_config& cfg, Params& P);

// The camera and the radiance-field parts; PG_ERR_ARG with a reason on a bad value.
pg_status camera_params(const pg_camera& cam, Params& P, std::string& why);
pg_status field_params(const pg_field* f, Params& P, std::string& why);

}  // namespace pgk
