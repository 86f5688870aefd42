// Engines for three-dimensional problems, degrees 1..2.
#include "batch.cuh"

namespace cutmg {

std::unique_ptr<EngineBase> make_engine_d3(int degree, const Hierarchy& H, cudaStream_t stream) {
  switch (degree) {
    case 1: return std::make_unique<Engine<3, 1>>(H, stream);
    case 2: return std::make_unique<Engine<3, 2>>(H, stream);
    default: throw std::invalid_argument("unsupported degree");
  }
}

std::unique_ptr<BatchGroupBase> make_batch_group_d3(int degree, const std::vector<EngineBase*>& inst,
                                                      int n_c) {
  switch (degree) {
    case 1: {
      std::vector<Engine<3, 1>*> v;
      for (EngineBase* e : inst) v.push_back(static_cast<Engine<3, 1>*>(e));
      return std::make_unique<BatchGroup<3, 1>>(v, n_c);
    }
    case 2: {
      std::vector<Engine<3, 2>*> v;
      for (EngineBase* e : inst) v.push_back(static_cast<Engine<3, 2>*>(e));
      return std::make_unique<BatchGroup<3, 2>>(v, n_c);
    }
    default: throw std::invalid_argument("unsupported degree");
  }
}

}  // namespace cutmg
