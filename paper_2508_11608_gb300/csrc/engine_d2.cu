// Engines for two-dimensional problems, degrees 1..4.
#include "batch.cuh"

namespace cutmg {

std::unique_ptr<EngineBase> make_engine_d2(int degree, const Hierarchy& H, cudaStream_t stream) {
  switch (degree) {
    case 1: return std::make_unique<Engine<2, 1>>(H, stream);
    case 2: return std::make_unique<Engine<2, 2>>(H, stream);
    case 3: return std::make_unique<Engine<2, 3>>(H, stream);
    case 4: return std::make_unique<Engine<2, 4>>(H, stream);
    default: throw std::invalid_argument("unsupported degree");
  }
}

std::unique_ptr<BatchGroupBase> make_batch_group_d2(int degree, const std::vector<EngineBase*>& inst,
                                                      int n_c) {
  switch (degree) {
    case 1: {
      std::vector<Engine<2, 1>*> v;
      for (EngineBase* e : inst) v.push_back(static_cast<Engine<2, 1>*>(e));
      return std::make_unique<BatchGroup<2, 1>>(v, n_c);
    }
    case 2: {
      std::vector<Engine<2, 2>*> v;
      for (EngineBase* e : inst) v.push_back(static_cast<Engine<2, 2>*>(e));
      return std::make_unique<BatchGroup<2, 2>>(v, n_c);
    }
    case 3: {
      std::vector<Engine<2, 3>*> v;
      for (EngineBase* e : inst) v.push_back(static_cast<Engine<2, 3>*>(e));
      return std::make_unique<BatchGroup<2, 3>>(v, n_c);
    }
    case 4: {
      std::vector<Engine<2, 4>*> v;
      for (EngineBase* e : inst) v.push_back(static_cast<Engine<2, 4>*>(e));
      return std::make_unique<BatchGroup<2, 4>>(v, n_c);
    }
    default: throw std::invalid_argument("unsupported degree");
  }
}

}  // namespace cutmg
