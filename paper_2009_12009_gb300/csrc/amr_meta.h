// amr_meta.h -- host tables of the two-level composite operator.
#pragma once

#include <string>
#include <vector>

#include "amr.h"
#include "meta.h"

namespace gmg {

struct AmrHost {
  std::vector<CfGhost> cf;
  std::vector<RefluxCell> rcells;
  std::vector<RefluxFace> rfaces;
  std::vector<unsigned char> covered;  // coarse level-0 layout
  std::vector<int64_t> covered_list;
  std::vector<int> cfidx;              // fine layout
  std::vector<AvgFace> avg_faces;
  std::vector<AvgCell> avg_cells;
};

// Tables of the composite operator for coarse level C (AMR level 0, MG level 0) and the
// finalized fine level F (allow_cf set).  Also sets F.parent (coarse box holding each fine
// box's coarsened image) and F.coarse_chunks.  Returns "" or an error message.
std::string build_amr(const LevelMeta& C, LevelMeta& F, AmrHost& A);

}  // namespace gmg
