"""GB300-native (sm_103a) renderer for rays through non-magnetic uniaxial
cylindrical invisibility cloaks (Halimeh & Wegener, arXiv:1209.6038)."""
