// Definitions of the opaque C ABI handles (shared by the ABI translation units).
#pragma once

#include <memory>

#include "factor.h"
#include "sgf.h"
#include "sgf_internal.h"

struct sgf_plan {
  sgf::Plan p;
};

struct sgf_factor_s {
  std::unique_ptr<sgf::FactorBase> f;
  const sgf_plan* plan;
};
