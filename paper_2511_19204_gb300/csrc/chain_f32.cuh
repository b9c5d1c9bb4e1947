// The lanes-per-chain rollout device functions in FP32 (the product): the bodies
// rollout_lanes.cuh and rollout_split.cuh instantiated with float in namespace mppi.
#pragma once
#include <type_traits>

#include "internal.h"
#include "rollout_warp.cuh"

#include "scalar_macros.h"
#include "rollout_lanes.cuh"
#include "rollout_split.cuh"
