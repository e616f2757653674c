"""Plain FP64 CPU oracle of the PIC/MCC timestep (test infrastructure only)."""
