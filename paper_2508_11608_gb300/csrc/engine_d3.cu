// Engines for three-dimensional problems, degrees 1..2.
#include "engine.cuh"

namespace cutmg {

std::unique_ptr<EngineBase> make_engine_d3(int degree, const Hierarchy& H) {
  switch (degree) {
    case 1: return std::make_unique<Engine<3, 1>>(H);
    case 2: return std::make_unique<Engine<3, 2>>(H);
    default: throw std::invalid_argument("unsupported degree");
  }
}

}  // namespace cutmg
