"""B300-native BML traffic cellular automaton (sm_103a CUDA behind a C ABI)."""
