// Engines for two-dimensional problems, degrees 1..3.
#include "engine.cuh"

namespace cutmg {

std::unique_ptr<EngineBase> make_engine_d2(int degree, const Hierarchy& H) {
  switch (degree) {
    case 1: return std::make_unique<Engine<2, 1>>(H);
    case 2: return std::make_unique<Engine<2, 2>>(H);
    case 3: return std::make_unique<Engine<2, 3>>(H);
    default: throw std::invalid_argument("unsupported degree");
  }
}

}  // namespace cutmg
