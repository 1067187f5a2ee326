"""FP64 CPU oracle for OSP / OSP-T. Test infrastructure only: the product path never imports it."""
