"""GB300 (sm_103a) isoperimetric clustering hot path (arXiv 1702.04739)."""
